/*
 * kg_oracle.c -- independent FP64 CPU oracle for the Fourier pseudo-spectral
 * solver of the real cubic Klein-Gordon equation
 *
 *     u_tt - Laplace(u) + u = |u|^2 u          (Aseeri et al., Eq. (1), section 1)
 *
 * stepped with the second-order semi-implicit scheme of section 1.1.2, Eq. (2),
 * in Fourier space with the nonlinear term formed in real space (section 1.1.2).
 *
 * TEST INFRASTRUCTURE. This file is the oracle the GPU library is checked against.
 * Only the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it. It shares no code, header, table or helper with the CUDA
 * library: it has its own textbook FFT, its own coefficients and its own sums.
 * Everything is plain IEEE double, evaluated in the order the formulas are written
 * (built with -ffp-contract=off so no fused multiply-add changes that order).
 * OpenMP only splits independent lines and independent modes across threads.
 *
 * Conventions (the paper fixes none of them; the readings below are the ones the
 * GPU library implements as well):
 *   grid        N^3 points on [-L/2, L/2)^3, x_j = -L/2 + j h, h = L/N; physical
 *               arrays are [z][y][x] with x fastest.
 *   transforms  forward DFT uh_k = sum_x u_x exp(-2 pi i m.j / N), unnormalised;
 *               inverse carries 1/N^3.  The real-to-complex half spectrum keeps
 *               kx = 0..N/2 and is stored [kz][ky][kx] with kx fastest.  In the
 *               complex-to-real inverse the kx = 0 and kx = N/2 entries contribute
 *               their real parts only (the imaginary part of each x-line result is
 *               discarded), i.e. the result is Re(ifftn(Hermitian extension)).
 *   wavenumbers m in FFT order {0..N/2-1, -N/2..-1}, k = 2 pi m / L,
 *               k^2 = kx^2 + ky^2 + kz^2; the Nyquist index keeps k^2 = (pi N/L)^2.
 *   nonlinearity F = lam * u^3 pointwise, no dealiasing (lam = 1 is Eq. (1) for real
 *               u; lam = 0 switches the nonlinearity off for closed-form tests).
 *   step        Eq. (2) in Fourier space, where Laplace -> -k^2 and omega^2 = 1 + k^2:
 *                 uh^{n+1} = 2 c_k uh^n - uh^{n-1} + 2 beta_k Fh^n,
 *                 c_k    = (1 - dt^2 omega^2 / 4) / (1 + dt^2 omega^2 / 4),
 *                 beta_k = (dt^2 / 2)            / (1 + dt^2 omega^2 / 4).
 *   startup     (the paper gives none) the symmetric fictitious level
 *                 uh^{-1} = c_k uh^0 - dt vh^0 + beta_k Fh^0,
 *               i.e. Eq. (2) at n = 0 with (u^1 - u^{-1}) / (2 dt) = v0.
 *   energy      (the paper gives the continuous functional of section 1.1 only)
 *                 Q^{n+1/2} = (h^3/N^3) sum_k w_k [ 1/2 |(uh^{n+1}-uh^n)/dt|^2
 *                                               + 1/2 omega_k^2 |(uh^{n+1}+uh^n)/2|^2 ]
 *                 P^n       = lam (h^3/4) sum_x (u^n)^4
 *                 E^{n+1/2} = Q^{n+1/2} - (P^n + P^{n+1}) / 2
 *               with w_k = 1 on the kx = 0 and kx = N/2 planes and 2 elsewhere
 *               (Parseval for a real field).  Q is exactly conserved by the linear
 *               scheme; all sums use Neumaier compensation.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "kg_oracle.h"

#define KGO_PI 3.14159265358979323846

typedef kgo_complex cplx;

static cplx c_add(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static cplx c_mul(cplx a, cplx b) {
    cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return r;
}

/* ---------------------------------------------------------------------------
 * Neumaier (improved Kahan-Babuska) compensated summation.
 * ------------------------------------------------------------------------- */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum* acc, double x) {
    double t = acc->s + x;
    if (fabs(acc->s) >= fabs(x)) acc->c += (acc->s - t) + x;
    else acc->c += (x - t) + acc->s;
    acc->s = t;
}
static double nsum_value(const nsum* acc) { return acc->s + acc->c; }

/* ---------------------------------------------------------------------------
 * 1D DFT: textbook recursive mixed-radix Cooley-Tukey, decimation in time.
 *
 * For n = p m with p the smallest prime factor of n, the input splits into the
 * p decimated subsequences x[r + p j] (j = 0..m-1); their length-m DFTs Y_r give
 *     X[k] = sum_{r=0}^{p-1} W_n^{r k} Y_r[k mod m],   W_n = exp(sign 2 pi i / n).
 * A prime n has p = n and m = 1, so the recursion ends in the direct DFT sum.
 * Twiddles come from a table of W_N^j for the top-level length N (libm cos/sin);
 * at a sub-length n, W_n^t = W_N^{t N / n}.
 * ------------------------------------------------------------------------- */
typedef struct {
    int n;
    cplx* tw;   /* tw[j] = exp(sign 2 pi i j / n) */
} dft_plan;

static int smallest_prime_factor(int n) {
    for (int p = 2; (long)p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

static int dft_plan_init(dft_plan* pl, int n, int sign) {
    pl->n = n;
    pl->tw = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    if (!pl->tw) return -1;
    for (int j = 0; j < n; j++) {
        double ang = 2.0 * KGO_PI * (double)j / (double)n;
        pl->tw[j].re = cos(ang);
        pl->tw[j].im = (double)sign * sin(ang);
    }
    return 0;
}
static void dft_plan_free(dft_plan* pl) { free(pl->tw); pl->tw = NULL; }

/* out and scratch: n entries each, disjoint.  x is read with stride s. */
static void dft_rec(const dft_plan* pl, int n, const cplx* x, ptrdiff_t s, cplx* out, cplx* scratch) {
    if (n == 1) { out[0] = x[0]; return; }
    int p = smallest_prime_factor(n);
    int m = n / p;
    int twstep = pl->n / n;
    /* sub-transform r lands in scratch[r m .. r m + m), using out[r m ..) as its scratch */
    for (int r = 0; r < p; r++) dft_rec(pl, m, x + r * s, s * p, scratch + (ptrdiff_t)r * m, out + (ptrdiff_t)r * m);
    for (int k = 0; k < n; k++) {
        cplx acc = {0.0, 0.0};
        for (int r = 0; r < p; r++) {
            long t = ((long)r * k) % n;
            acc = c_add(acc, c_mul(pl->tw[t * twstep], scratch[(ptrdiff_t)r * m + k % m]));
        }
        out[k] = acc;
    }
}

int kgo_dft1d(int n, int sign, const kgo_complex* in, ptrdiff_t istride, kgo_complex* out) {
    if (n < 1 || (sign != 1 && sign != -1)) return -1;
    dft_plan pl;
    if (dft_plan_init(&pl, n, sign)) return -2;
    cplx* scratch = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    if (!scratch) { dft_plan_free(&pl); return -2; }
    dft_rec(&pl, n, in, istride, out, scratch);
    free(scratch);
    dft_plan_free(&pl);
    return 0;
}

/* ---------------------------------------------------------------------------
 * 3D real-to-complex / complex-to-real transforms on the N^3 grid.
 * Spectral array: [kz][ky][kx], kx = 0..N/2 fastest, NH = N/2 + 1.
 * ------------------------------------------------------------------------- */
static size_t spec_len(int N) { return (size_t)N * N * (size_t)(N / 2 + 1); }

/* complex DFT along y (axis 1) or z (axis 2) of every line of a spectral array */
static int fft_axis_yz(int N, cplx* a, int axis, int sign) {
    const int NH = N / 2 + 1;
    dft_plan pl;
    if (dft_plan_init(&pl, N, sign)) return -2;
    int err = 0;
    /* lines: axis 1 -> (z, kx) pairs, stride NH; axis 2 -> (y, kx) pairs, stride N NH */
    const ptrdiff_t stride = (axis == 1) ? NH : (ptrdiff_t)N * NH;
    const long nlines = (long)N * NH;
#pragma omp parallel
    {
        cplx* in = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        cplx* scr = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        if (!in || !out || !scr) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (long line = 0; line < nlines; line++) {
                long outer = line / NH, kx = line % NH;
                ptrdiff_t base = (axis == 1) ? (ptrdiff_t)outer * N * NH + kx : (ptrdiff_t)outer * NH + kx;
                for (int j = 0; j < N; j++) in[j] = a[base + (ptrdiff_t)j * stride];
                dft_rec(&pl, N, in, 1, out, scr);
                for (int j = 0; j < N; j++) a[base + (ptrdiff_t)j * stride] = out[j];
            }
        }
        free(in); free(out); free(scr);
    }
    dft_plan_free(&pl);
    return err;
}

int kgo_fft_axis(int N, kgo_complex* a, int axis, int sign) {
    if (N < 2 || (N & 1) || (axis != 1 && axis != 2) || (sign != 1 && sign != -1)) return -1;
    return fft_axis_yz(N, a, axis, sign);
}

/* forward real-to-complex DFT of every x-line: out[z][y][kx], kx = 0..N/2 */
int kgo_r2c_x(int N, const double* u, kgo_complex* out) {
    if (N < 2 || (N & 1)) return -1;
    const int NH = N / 2 + 1;
    dft_plan pl;
    if (dft_plan_init(&pl, N, -1)) return -2;
    int err = 0;
    const long nlines = (long)N * N;
#pragma omp parallel
    {
        cplx* in = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        cplx* res = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        cplx* scr = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        if (!in || !res || !scr) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (long line = 0; line < nlines; line++) {
                for (int j = 0; j < N; j++) { in[j].re = u[line * N + j]; in[j].im = 0.0; }
                dft_rec(&pl, N, in, 1, res, scr);
                for (int k = 0; k < NH; k++) out[line * NH + k] = res[k];
            }
        }
        free(in); free(res); free(scr);
    }
    dft_plan_free(&pl);
    return err;
}

/* inverse DFT of every x-line of a half spectrum, real part only, times scale.
 * The length-N line is the Hermitian extension X[N-k] = conj(X[k]) (0 < k < N/2);
 * X[0] and X[N/2] enter as stored and the imaginary part of the result is dropped. */
int kgo_c2r_x(int N, const kgo_complex* in, double* u, double scale) {
    if (N < 2 || (N & 1)) return -1;
    const int NH = N / 2 + 1;
    dft_plan pl;
    if (dft_plan_init(&pl, N, +1)) return -2;
    int err = 0;
    const long nlines = (long)N * N;
#pragma omp parallel
    {
        cplx* full = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        cplx* res = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        cplx* scr = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        if (!full || !res || !scr) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (long line = 0; line < nlines; line++) {
                const cplx* X = in + line * NH;
                for (int k = 0; k < NH; k++) full[k] = X[k];
                for (int k = 1; k < N / 2; k++) { full[N - k].re = X[k].re; full[N - k].im = -X[k].im; }
                dft_rec(&pl, N, full, 1, res, scr);
                for (int j = 0; j < N; j++) u[line * N + j] = res[j].re * scale;
            }
        }
        free(full); free(res); free(scr);
    }
    dft_plan_free(&pl);
    return err;
}

int kgo_r2c3d(int N, const double* u, kgo_complex* uh) {
    int e = kgo_r2c_x(N, u, uh);
    if (!e) e = fft_axis_yz(N, uh, 1, -1);
    if (!e) e = fft_axis_yz(N, uh, 2, -1);
    return e;
}

/* uh is left untouched; tmp-free by working on a private copy */
int kgo_c2r3d(int N, const kgo_complex* uh, double* u) {
    if (N < 2 || (N & 1)) return -1;
    size_t len = spec_len(N);
    cplx* w = (cplx*)malloc(sizeof(cplx) * len);
    if (!w) return -2;
    memcpy(w, uh, sizeof(cplx) * len);
    int e = fft_axis_yz(N, w, 2, +1);
    if (!e) e = fft_axis_yz(N, w, 1, +1);
    if (!e) e = kgo_c2r_x(N, w, u, 1.0 / ((double)N * (double)N * (double)N));
    free(w);
    return e;
}

/* ---------------------------------------------------------------------------
 * Wavenumbers and coefficients of Eq. (2) in Fourier space.
 * ------------------------------------------------------------------------- */
static long fft_index_to_m(long j, int N) { return (j <= N / 2) ? j : j - N; }

/* k^2 of the mode stored at [kz][ky][kx] (kx = 0..N/2) */
static double mode_k2(int N, double L, long kz, long ky, long kx) {
    long mz = fft_index_to_m(kz, N), my = fft_index_to_m(ky, N), mx = kx;
    double kfac = 2.0 * KGO_PI / L;
    double kzv = kfac * (double)mz, kyv = kfac * (double)my, kxv = kfac * (double)mx;
    return kxv * kxv + kyv * kyv + kzv * kzv;
}

static void scheme_coeffs(double dt, double k2, double* c, double* beta, double* omega2) {
    double w2 = 1.0 + k2;
    double a = dt * dt * w2 / 4.0;
    *c = (1.0 - a) / (1.0 + a);
    *beta = (dt * dt / 2.0) / (1.0 + a);
    *omega2 = w2;
}

int kgo_coeffs(double dt, double k2, double* c, double* beta) {
    double w2;
    scheme_coeffs(dt, k2, c, beta, &w2);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Spectral derivative (tests): multiply by (i kx)^ox (i ky)^oy (i kz)^oz.
 * An odd order along an axis zeroes that axis' Nyquist index (its derivative of
 * the real cosine at m = -N/2 is not representable); even orders keep it.
 * ------------------------------------------------------------------------- */
int kgo_spectral_deriv(int N, double L, const double* u, int ox, int oy, int oz, double* out) {
    if (N < 2 || (N & 1) || ox < 0 || oy < 0 || oz < 0) return -1;
    const int NH = N / 2 + 1;
    size_t len = spec_len(N);
    cplx* uh = (cplx*)malloc(sizeof(cplx) * len);
    if (!uh) return -2;
    int e = kgo_r2c3d(N, u, uh);
    if (e) { free(uh); return e; }
    const double kfac = 2.0 * KGO_PI / L;
#pragma omp parallel for schedule(static)
    for (long kz = 0; kz < N; kz++)
        for (long ky = 0; ky < N; ky++)
            for (long kx = 0; kx < NH; kx++) {
                long m[3] = {kx, fft_index_to_m(ky, N), fft_index_to_m(kz, N)};
                int ord[3] = {ox, oy, oz};
                cplx fac = {1.0, 0.0};
                for (int ax = 0; ax < 3; ax++) {
                    if ((ord[ax] & 1) && (m[ax] == N / 2 || m[ax] == -N / 2)) { fac.re = 0.0; fac.im = 0.0; }
                    cplx ik = {0.0, kfac * (double)m[ax]};
                    for (int q = 0; q < ord[ax]; q++) fac = c_mul(fac, ik);
                }
                size_t idx = ((size_t)kz * N + ky) * NH + kx;
                uh[idx] = c_mul(fac, uh[idx]);
            }
    e = kgo_c2r3d(N, uh, out);
    free(uh);
    return e;
}

/* ---------------------------------------------------------------------------
 * Solver state.
 * ------------------------------------------------------------------------- */
struct kgo_state {
    int N;
    double L, dt, lam;
    long level;        /* n */
    cplx* a;           /* uh^n     */
    cplx* b;           /* uh^{n-1} */
    cplx* f;           /* spectral scratch */
    double* u;         /* physical scratch */
    double last_maxabs;
};

static void state_free(kgo_state* s) {
    if (!s) return;
    free(s->a); free(s->b); free(s->f); free(s->u);
    free(s);
}

void kgo_destroy(kgo_state* s) { state_free(s); }

/* Fh = R2C(lam u^3) from the physical field in s->u; also returns max |u| */
static int nonlinear_hat(kgo_state* s, double* maxabs) {
    const size_t n3 = (size_t)s->N * s->N * s->N;
    double mx = 0.0;
    double lam = s->lam;
    double* u = s->u;
#pragma omp parallel for schedule(static) reduction(max : mx)
    for (size_t i = 0; i < n3; i++) {
        double v = u[i];
        double av = fabs(v);
        if (av > mx || av != av) mx = (av != av) ? INFINITY : av;
        u[i] = lam * (v * v * v);
    }
    if (maxabs) *maxabs = mx;
    return kgo_r2c3d(s->N, u, s->f);
}

kgo_state* kgo_create(int N, double L, double dt, double lam, const double* u0, const double* v0) {
    if (N < 2 || (N & 1) || !(L > 0.0) || !(dt > 0.0) || !u0) return NULL;
    kgo_state* s = (kgo_state*)calloc(1, sizeof(kgo_state));
    if (!s) return NULL;
    s->N = N; s->L = L; s->dt = dt; s->lam = lam; s->level = 0;
    const size_t len = spec_len(N), n3 = (size_t)N * N * N;
    s->a = (cplx*)malloc(sizeof(cplx) * len);
    s->b = (cplx*)malloc(sizeof(cplx) * len);
    s->f = (cplx*)malloc(sizeof(cplx) * len);
    s->u = (double*)malloc(sizeof(double) * n3);
    if (!s->a || !s->b || !s->f || !s->u) { state_free(s); return NULL; }

    /* uh^0 */
    if (kgo_r2c3d(N, u0, s->a)) { state_free(s); return NULL; }
    /* vh^0 (kept in b until the startup formula overwrites it) */
    if (v0) {
        if (kgo_r2c3d(N, v0, s->b)) { state_free(s); return NULL; }
    } else {
        memset(s->b, 0, sizeof(cplx) * len);
    }
    /* Fh^0 */
    memcpy(s->u, u0, sizeof(double) * n3);
    if (nonlinear_hat(s, &s->last_maxabs)) { state_free(s); return NULL; }

    /* uh^{-1} = c_k uh^0 - dt vh^0 + beta_k Fh^0 */
    const int NH = N / 2 + 1;
#pragma omp parallel for schedule(static)
    for (long kz = 0; kz < N; kz++)
        for (long ky = 0; ky < N; ky++)
            for (long kx = 0; kx < NH; kx++) {
                size_t i = ((size_t)kz * N + ky) * NH + kx;
                double c, beta, w2;
                scheme_coeffs(dt, mode_k2(N, L, kz, ky, kx), &c, &beta, &w2);
                cplx a0 = s->a[i], v = s->b[i], f = s->f[i];
                s->b[i].re = c * a0.re - dt * v.re + beta * f.re;
                s->b[i].im = c * a0.im - dt * v.im + beta * f.im;
            }
    return s;
}

int kgo_step(kgo_state* s, int nsteps, double threshold, long* blowup_level) {
    if (!s || nsteps < 0) return -1;
    const int N = s->N, NH = N / 2 + 1;
    for (int it = 0; it < nsteps; it++) {
        /* u^n in physical space, then Fh^n = R2C(lam (u^n)^3) */
        if (kgo_c2r3d(N, s->a, s->u)) return -2;
        double mx;
        if (nonlinear_hat(s, &mx)) return -2;
        s->last_maxabs = mx;
        if (threshold > 0.0 && !(mx <= threshold)) {   /* blow-up: freeze at this level */
            if (blowup_level) *blowup_level = s->level;
            return 1;
        }
        /* uh^{n+1} = 2 c_k uh^n - uh^{n-1} + 2 beta_k Fh^n, written over uh^{n-1} */
#pragma omp parallel for schedule(static)
        for (long kz = 0; kz < N; kz++)
            for (long ky = 0; ky < N; ky++)
                for (long kx = 0; kx < NH; kx++) {
                    size_t i = ((size_t)kz * N + ky) * NH + kx;
                    double c, beta, w2;
                    scheme_coeffs(s->dt, mode_k2(N, s->L, kz, ky, kx), &c, &beta, &w2);
                    cplx an = s->a[i], bn = s->b[i], f = s->f[i];
                    s->b[i].re = 2.0 * c * an.re - bn.re + 2.0 * beta * f.re;
                    s->b[i].im = 2.0 * c * an.im - bn.im + 2.0 * beta * f.im;
                }
        cplx* t = s->a; s->a = s->b; s->b = t;
        s->level++;
    }
    return 0;
}

long kgo_level(const kgo_state* s) { return s ? s->level : -1; }
double kgo_last_maxabs(const kgo_state* s) { return s ? s->last_maxabs : NAN; }

int kgo_fetch(const kgo_state* s, double* u) {
    if (!s || !u) return -1;
    return kgo_c2r3d(s->N, s->a, u);
}

int kgo_fetch_spectral(const kgo_state* s, kgo_complex* a, kgo_complex* b) {
    if (!s) return -1;
    size_t len = spec_len(s->N);
    if (a) memcpy(a, s->a, sizeof(cplx) * len);
    if (b) memcpy(b, s->b, sizeof(cplx) * len);
    return 0;
}

/* Q(x, y) = (h^3/N^3) sum_k w_k [1/2 |(x - y)/dt|^2 + 1/2 omega^2 |(x + y)/2|^2] */
static double quadratic_energy(int N, double L, double dt, const cplx* x, const cplx* y) {
    const int NH = N / 2 + 1;
    const double h = L / (double)N;
    const double norm = h * h * h / ((double)N * (double)N * (double)N);
    nsum total = {0.0, 0.0};
    /* per-plane compensated partials, combined serially in plane order */
    double* part_s = (double*)calloc((size_t)N, sizeof(double));
    double* part_c = (double*)calloc((size_t)N, sizeof(double));
    if (!part_s || !part_c) { free(part_s); free(part_c); return NAN; }
#pragma omp parallel for schedule(static)
    for (long kz = 0; kz < N; kz++) {
        nsum acc = {0.0, 0.0};
        for (long ky = 0; ky < N; ky++)
            for (long kx = 0; kx < NH; kx++) {
                size_t i = ((size_t)kz * N + ky) * NH + kx;
                double w = (kx == 0 || kx == N / 2) ? 1.0 : 2.0;
                double c, beta, w2;
                scheme_coeffs(dt, mode_k2(N, L, kz, ky, kx), &c, &beta, &w2);
                double dre = (x[i].re - y[i].re) / dt, dim = (x[i].im - y[i].im) / dt;
                double sre = (x[i].re + y[i].re) / 2.0, sim = (x[i].im + y[i].im) / 2.0;
                double term = 0.5 * (dre * dre + dim * dim) + 0.5 * w2 * (sre * sre + sim * sim);
                nsum_add(&acc, w * term);
            }
        part_s[kz] = acc.s;
        part_c[kz] = acc.c;
    }
    for (long kz = 0; kz < N; kz++) { nsum_add(&total, part_s[kz]); nsum_add(&total, part_c[kz]); }
    free(part_s); free(part_c);
    return norm * nsum_value(&total);
}

/* P = lam (h^3/4) sum_x u^4 */
static double quartic_energy(int N, double L, double lam, const double* u) {
    const double h = L / (double)N;
    nsum total = {0.0, 0.0};
    double* part_s = (double*)calloc((size_t)N, sizeof(double));
    double* part_c = (double*)calloc((size_t)N, sizeof(double));
    if (!part_s || !part_c) { free(part_s); free(part_c); return NAN; }
    const size_t plane = (size_t)N * N;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < N; z++) {
        nsum acc = {0.0, 0.0};
        for (size_t i = 0; i < plane; i++) {
            double v = u[z * plane + i];
            double v2 = v * v;
            nsum_add(&acc, v2 * v2);
        }
        part_s[z] = acc.s;
        part_c[z] = acc.c;
    }
    for (long z = 0; z < N; z++) { nsum_add(&total, part_s[z]); nsum_add(&total, part_c[z]); }
    free(part_s); free(part_c);
    return lam * (h * h * h / 4.0) * nsum_value(&total);
}

int kgo_energy_parts(kgo_state* s, double* Q, double* Pn, double* Pnm1) {
    if (!s) return -1;
    const int N = s->N;
    if (Q) *Q = quadratic_energy(N, s->L, s->dt, s->a, s->b);
    if (Pn) {
        if (kgo_c2r3d(N, s->a, s->u)) return -2;
        *Pn = quartic_energy(N, s->L, s->lam, s->u);
    }
    if (Pnm1) {
        if (kgo_c2r3d(N, s->b, s->u)) return -2;
        *Pnm1 = quartic_energy(N, s->L, s->lam, s->u);
    }
    return 0;
}

/* E^{n-1/2} at level n */
int kgo_energy(kgo_state* s, double* E) {
    double Q, Pn, Pm;
    int e = kgo_energy_parts(s, &Q, &Pn, &Pm);
    if (e) return e;
    *E = Q - 0.5 * (Pn + Pm);
    return 0;
}

/* Continuous energy of (u0, v0) at t = 0 with the gradient taken spectrally:
 * h^3 sum [v0^2/2 + u0^2/2 - lam u0^4/4] + (h^3/N^3) sum_k w_k k^2 |uh0|^2 / 2 */
int kgo_energy_initial(int N, double L, double lam, const double* u0, const double* v0, double* E) {
    if (N < 2 || (N & 1) || !u0 || !E) return -1;
    const int NH = N / 2 + 1;
    const double h = L / (double)N;
    const size_t n3 = (size_t)N * N * N, len = spec_len(N);
    nsum acc = {0.0, 0.0};
    for (size_t i = 0; i < n3; i++) {
        double u = u0[i], v = v0 ? v0[i] : 0.0;
        nsum_add(&acc, h * h * h * (0.5 * v * v + 0.5 * u * u - lam * 0.25 * u * u * u * u));
    }
    cplx* uh = (cplx*)malloc(sizeof(cplx) * len);
    if (!uh) return -2;
    if (kgo_r2c3d(N, u0, uh)) { free(uh); return -2; }
    const double norm = h * h * h / ((double)N * (double)N * (double)N);
    for (long kz = 0; kz < N; kz++)
        for (long ky = 0; ky < N; ky++)
            for (long kx = 0; kx < NH; kx++) {
                size_t i = ((size_t)kz * N + ky) * NH + kx;
                double w = (kx == 0 || kx == N / 2) ? 1.0 : 2.0;
                double k2 = mode_k2(N, L, kz, ky, kx);
                nsum_add(&acc, norm * w * 0.5 * k2 * (uh[i].re * uh[i].re + uh[i].im * uh[i].im));
            }
    free(uh);
    *E = nsum_value(&acc);
    return 0;
}

/* Low-mode shell energies of u0 (learned-ranker features):
 *   E_j = (h^3/N^3) sum_{k in shell j} w_k omega_k^2 |uh0_k|^2 / 2,
 * shells by integer wavenumber norm |m|: {0}, (0,1], (1,2], (2,4]. */
int kgo_shell_energies(int N, double L, const double* u0, double* out4) {
    if (N < 2 || (N & 1) || !u0 || !out4) return -1;
    const int NH = N / 2 + 1;
    const double h = L / (double)N;
    const size_t len = spec_len(N);
    cplx* uh = (cplx*)malloc(sizeof(cplx) * len);
    if (!uh) return -2;
    if (kgo_r2c3d(N, u0, uh)) { free(uh); return -2; }
    const double norm = h * h * h / ((double)N * (double)N * (double)N);
    nsum sh[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (long kz = 0; kz < N; kz++)
        for (long ky = 0; ky < N; ky++)
            for (long kx = 0; kx < NH; kx++) {
                long mz = fft_index_to_m(kz, N), my = fft_index_to_m(ky, N), mx = kx;
                long m2 = mx * mx + my * my + mz * mz;
                int j = (m2 == 0) ? 0 : (m2 <= 1) ? 1 : (m2 <= 4) ? 2 : (m2 <= 16) ? 3 : -1;
                if (j < 0) continue;
                size_t i = ((size_t)kz * N + ky) * NH + kx;
                double w = (kx == 0 || kx == N / 2) ? 1.0 : 2.0;
                double w2 = 1.0 + mode_k2(N, L, kz, ky, kx);
                nsum_add(&sh[j], norm * w * 0.5 * w2 * (uh[i].re * uh[i].re + uh[i].im * uh[i].im));
            }
    for (int j = 0; j < 4; j++) out4[j] = nsum_value(&sh[j]);
    free(uh);
    return 0;
}

int kgo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void kgo_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------
 * Complex field (section 1.1.2 notes that the implementation allows a complex
 * u; Eq. (1) is written with |u|^2 u).  Same scheme, same coefficients; the
 * field is complex, so the spectrum is the full N^3 array [kz][ky][kx] with
 * kx = 0..N-1 in FFT order, no Hermitian symmetry and no C2R rule:
 *   nonlinearity F = lam |u|^2 u
 *   energy       Q^{n+1/2} = (h^3/N^3) sum_k [ 1/2 |(uh^{n+1}-uh^n)/dt|^2
 *                                         + 1/2 omega_k^2 |(uh^{n+1}+uh^n)/2|^2 ]
 *                P^n = lam (h^3/4) sum_x |u^n|^4   (every mode has weight 1)
 * For a real u these are the real-field definitions above (Parseval).
 * ------------------------------------------------------------------------- */

/* complex DFT along axis 0 (x), 1 (y) or 2 (z) of every line of an N^3 array */
static int fft_axis_full(int N, cplx* a, int axis, int sign) {
    dft_plan pl;
    if (dft_plan_init(&pl, N, sign)) return -2;
    int err = 0;
    const ptrdiff_t stride = (axis == 0) ? 1 : (axis == 1) ? (ptrdiff_t)N : (ptrdiff_t)N * N;
    const long nlines = (long)N * N;
#pragma omp parallel
    {
        cplx* in = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        cplx* scr = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        if (!in || !out || !scr) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (long line = 0; line < nlines; line++) {
                long hi = line / N, lo = line % N;   /* the two indices other than the axis */
                ptrdiff_t base;
                if (axis == 0) base = (ptrdiff_t)line * N;                       /* (z, y) */
                else if (axis == 1) base = (ptrdiff_t)hi * N * N + lo;           /* (z, x) */
                else base = (ptrdiff_t)hi * N + lo;                              /* (y, x) */
                for (int j = 0; j < N; j++) in[j] = a[base + (ptrdiff_t)j * stride];
                dft_rec(&pl, N, in, 1, out, scr);
                for (int j = 0; j < N; j++) a[base + (ptrdiff_t)j * stride] = out[j];
            }
        }
        free(in); free(out); free(scr);
    }
    dft_plan_free(&pl);
    return err;
}

/* full 3D DFT in place, unnormalised (sign -1 forward, +1 inverse) */
int kgo_fft3d(int N, kgo_complex* a, int sign) {
    if (N < 2 || (N & 1) || (sign != 1 && sign != -1) || !a) return -1;
    for (int axis = 0; axis < 3; axis++) {
        int e = fft_axis_full(N, a, axis, sign);
        if (e) return e;
    }
    return 0;
}

/* k^2 of the mode stored at [kz][ky][kx] of the full spectrum */
static double mode_k2_full(int N, double L, long kz, long ky, long kx) {
    long mz = fft_index_to_m(kz, N), my = fft_index_to_m(ky, N), mx = fft_index_to_m(kx, N);
    double kfac = 2.0 * KGO_PI / L;
    double kzv = kfac * (double)mz, kyv = kfac * (double)my, kxv = kfac * (double)mx;
    return kxv * kxv + kyv * kyv + kzv * kzv;
}

struct kgoc_state {
    int N;
    double L, dt, lam;
    long level;
    cplx* a;      /* uh^n */
    cplx* b;      /* uh^{n-1} */
    cplx* f;      /* scratch: u^n, then F^n, then Fh^n */
    double last_maxabs;
};

void kgoc_destroy(kgoc_state* s) {
    if (!s) return;
    free(s->a); free(s->b); free(s->f);
    free(s);
}

/* u = ifft3d(x) / N^3 into s->f */
static int field_of(kgoc_state* s, const cplx* x) {
    const int N = s->N;
    const size_t n3 = (size_t)N * N * N;
    memcpy(s->f, x, sizeof(cplx) * n3);
    int e = kgo_fft3d(N, s->f, +1);
    if (e) return e;
    const double inv = 1.0 / ((double)N * (double)N * (double)N);
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < n3; i++) {
        s->f[i].re *= inv;
        s->f[i].im *= inv;
    }
    return 0;
}

/* s->f holds u: replace it by Fh = fft3d(lam |u|^2 u); max |u| into *maxabs */
static int nonlinear_hat_c(kgoc_state* s, double* maxabs) {
    const size_t n3 = (size_t)s->N * s->N * s->N;
    double mx = 0.0;
    const double lam = s->lam;
#pragma omp parallel for schedule(static) reduction(max : mx)
    for (size_t i = 0; i < n3; i++) {
        cplx v = s->f[i];
        double m2 = v.re * v.re + v.im * v.im;
        double av = sqrt(m2);
        if (av > mx || av != av) mx = (av != av) ? INFINITY : av;
        s->f[i].re = lam * (m2 * v.re);
        s->f[i].im = lam * (m2 * v.im);
    }
    if (maxabs) *maxabs = mx;
    return kgo_fft3d(s->N, s->f, -1);
}

kgoc_state* kgoc_create(int N, double L, double dt, double lam, const kgo_complex* u0, const kgo_complex* v0) {
    if (N < 2 || (N & 1) || !(L > 0.0) || !(dt > 0.0) || !u0) return NULL;
    kgoc_state* s = (kgoc_state*)calloc(1, sizeof(kgoc_state));
    if (!s) return NULL;
    s->N = N; s->L = L; s->dt = dt; s->lam = lam; s->level = 0;
    const size_t n3 = (size_t)N * N * N;
    s->a = (cplx*)malloc(sizeof(cplx) * n3);
    s->b = (cplx*)malloc(sizeof(cplx) * n3);
    s->f = (cplx*)malloc(sizeof(cplx) * n3);
    if (!s->a || !s->b || !s->f) { kgoc_destroy(s); return NULL; }
    memcpy(s->a, u0, sizeof(cplx) * n3);                        /* uh^0 */
    if (kgo_fft3d(N, s->a, -1)) { kgoc_destroy(s); return NULL; }
    if (v0) {                                                   /* vh^0, in b for now */
        memcpy(s->b, v0, sizeof(cplx) * n3);
        if (kgo_fft3d(N, s->b, -1)) { kgoc_destroy(s); return NULL; }
    } else {
        memset(s->b, 0, sizeof(cplx) * n3);
    }
    memcpy(s->f, u0, sizeof(cplx) * n3);                        /* Fh^0 */
    if (nonlinear_hat_c(s, &s->last_maxabs)) { kgoc_destroy(s); return NULL; }
    /* uh^{-1} = c_k uh^0 - dt vh^0 + beta_k Fh^0 */
#pragma omp parallel for schedule(static)
    for (long kz = 0; kz < N; kz++)
        for (long ky = 0; ky < N; ky++)
            for (long kx = 0; kx < N; kx++) {
                size_t i = ((size_t)kz * N + ky) * N + kx;
                double c, beta, w2;
                scheme_coeffs(dt, mode_k2_full(N, L, kz, ky, kx), &c, &beta, &w2);
                cplx a0 = s->a[i], v = s->b[i], f = s->f[i];
                s->b[i].re = c * a0.re - dt * v.re + beta * f.re;
                s->b[i].im = c * a0.im - dt * v.im + beta * f.im;
            }
    return s;
}

int kgoc_step(kgoc_state* s, int nsteps, double threshold, long* blowup_level) {
    if (!s || nsteps < 0) return -1;
    const int N = s->N;
    for (int it = 0; it < nsteps; it++) {
        if (field_of(s, s->a)) return -2;                      /* u^n */
        double mx;
        if (nonlinear_hat_c(s, &mx)) return -2;                /* Fh^n */
        s->last_maxabs = mx;
        if (threshold > 0.0 && !(mx <= threshold)) {
            if (blowup_level) *blowup_level = s->level;
            return 1;
        }
#pragma omp parallel for schedule(static)
        for (long kz = 0; kz < N; kz++)
            for (long ky = 0; ky < N; ky++)
                for (long kx = 0; kx < N; kx++) {
                    size_t i = ((size_t)kz * N + ky) * N + kx;
                    double c, beta, w2;
                    scheme_coeffs(s->dt, mode_k2_full(N, s->L, kz, ky, kx), &c, &beta, &w2);
                    cplx an = s->a[i], bn = s->b[i], f = s->f[i];
                    s->b[i].re = 2.0 * c * an.re - bn.re + 2.0 * beta * f.re;
                    s->b[i].im = 2.0 * c * an.im - bn.im + 2.0 * beta * f.im;
                }
        cplx* t = s->a; s->a = s->b; s->b = t;
        s->level++;
    }
    return 0;
}

long kgoc_level(const kgoc_state* s) { return s ? s->level : -1; }
double kgoc_last_maxabs(const kgoc_state* s) { return s ? s->last_maxabs : NAN; }

int kgoc_fetch(kgoc_state* s, kgo_complex* u) {
    if (!s || !u) return -1;
    int e = field_of(s, s->a);
    if (e) return e;
    memcpy(u, s->f, sizeof(cplx) * (size_t)s->N * s->N * s->N);
    return 0;
}

int kgoc_fetch_spectral(const kgoc_state* s, kgo_complex* a, kgo_complex* b) {
    if (!s) return -1;
    const size_t n3 = (size_t)s->N * s->N * s->N;
    if (a) memcpy(a, s->a, sizeof(cplx) * n3);
    if (b) memcpy(b, s->b, sizeof(cplx) * n3);
    return 0;
}

/* Q over the full spectrum, every mode weight 1 */
static double quadratic_energy_full(int N, double L, double dt, const cplx* x, const cplx* y) {
    const double h = L / (double)N;
    const double norm = h * h * h / ((double)N * (double)N * (double)N);
    nsum total = {0.0, 0.0};
    double* part_s = (double*)calloc((size_t)N, sizeof(double));
    double* part_c = (double*)calloc((size_t)N, sizeof(double));
    if (!part_s || !part_c) { free(part_s); free(part_c); return NAN; }
#pragma omp parallel for schedule(static)
    for (long kz = 0; kz < N; kz++) {
        nsum acc = {0.0, 0.0};
        for (long ky = 0; ky < N; ky++)
            for (long kx = 0; kx < N; kx++) {
                size_t i = ((size_t)kz * N + ky) * N + kx;
                double c, beta, w2;
                scheme_coeffs(dt, mode_k2_full(N, L, kz, ky, kx), &c, &beta, &w2);
                double dre = (x[i].re - y[i].re) / dt, dim = (x[i].im - y[i].im) / dt;
                double sre = (x[i].re + y[i].re) / 2.0, sim = (x[i].im + y[i].im) / 2.0;
                nsum_add(&acc, 0.5 * (dre * dre + dim * dim) + 0.5 * w2 * (sre * sre + sim * sim));
            }
        part_s[kz] = acc.s;
        part_c[kz] = acc.c;
    }
    for (long kz = 0; kz < N; kz++) { nsum_add(&total, part_s[kz]); nsum_add(&total, part_c[kz]); }
    free(part_s); free(part_c);
    return norm * nsum_value(&total);
}

/* P = lam (h^3/4) sum_x |u|^4 of the complex field in u */
static double quartic_energy_c(int N, double L, double lam, const cplx* u) {
    const double h = L / (double)N;
    nsum total = {0.0, 0.0};
    double* part_s = (double*)calloc((size_t)N, sizeof(double));
    double* part_c = (double*)calloc((size_t)N, sizeof(double));
    if (!part_s || !part_c) { free(part_s); free(part_c); return NAN; }
    const size_t plane = (size_t)N * N;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < N; z++) {
        nsum acc = {0.0, 0.0};
        for (size_t i = 0; i < plane; i++) {
            cplx v = u[z * plane + i];
            double m2 = v.re * v.re + v.im * v.im;
            nsum_add(&acc, m2 * m2);
        }
        part_s[z] = acc.s;
        part_c[z] = acc.c;
    }
    for (long z = 0; z < N; z++) { nsum_add(&total, part_s[z]); nsum_add(&total, part_c[z]); }
    free(part_s); free(part_c);
    return lam * (h * h * h / 4.0) * nsum_value(&total);
}

int kgoc_energy_parts(kgoc_state* s, double* Q, double* Pn, double* Pnm1) {
    if (!s) return -1;
    const int N = s->N;
    if (Q) *Q = quadratic_energy_full(N, s->L, s->dt, s->a, s->b);
    if (Pn) {
        if (field_of(s, s->a)) return -2;
        *Pn = quartic_energy_c(N, s->L, s->lam, s->f);
    }
    if (Pnm1) {
        if (field_of(s, s->b)) return -2;
        *Pnm1 = quartic_energy_c(N, s->L, s->lam, s->f);
    }
    return 0;
}

int kgoc_energy(kgoc_state* s, double* E) {
    double Q, Pn, Pm;
    int e = kgoc_energy_parts(s, &Q, &Pn, &Pm);
    if (e) return e;
    *E = Q - 0.5 * (Pn + Pm);
    return 0;
}
