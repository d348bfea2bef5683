/*
 * kg_oracle.h -- FP64 CPU oracle for the cubic Klein-Gordon Fourier spectral
 * scheme (Aseeri et al., Eq. (1) and Eq. (2), sections 1.1 and 1.1.2).
 *
 * TEST INFRASTRUCTURE: loaded only by the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark.  It shares nothing with the CUDA library.
 * All conventions (grid, transform signs, half-spectrum layout, C2R rule, Nyquist,
 * startup level, discrete energy) are stated at the top of kg_oracle.c.
 *
 * Return codes: 0 success, -1 invalid argument, -2 allocation failure.
 */
#ifndef KG_ORACLE_H
#define KG_ORACLE_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } kgo_complex;
typedef struct kgo_state kgo_state;

/* 1D DFT of length n (any n >= 1), sign -1 forward / +1 inverse, unnormalised.
 * in is read with stride istride; out is contiguous. */
int kgo_dft1d(int n, int sign, const kgo_complex* in, ptrdiff_t istride, kgo_complex* out);

/* 3D transforms on an N^3 grid (N even).  Half spectrum [kz][ky][kx], kx = 0..N/2. */
int kgo_r2c3d(int N, const double* u, kgo_complex* uh);          /* forward, unnormalised */
int kgo_c2r3d(int N, const kgo_complex* uh, double* u);          /* inverse, 1/N^3, Re only */

/* single-axis pieces of the 3D transforms */
int kgo_r2c_x(int N, const double* u, kgo_complex* out);                 /* every x-line, forward */
int kgo_c2r_x(int N, const kgo_complex* in, double* u, double scale);   /* every x-line, inverse, Re * scale */
int kgo_fft_axis(int N, kgo_complex* a, int axis, int sign);            /* axis 1 = y, 2 = z, in place */

/* scheme coefficients c_k, beta_k of Eq. (2) for a given k^2 */
int kgo_coeffs(double dt, double k2, double* c, double* beta);

/* spectral derivative (i kx)^ox (i ky)^oy (i kz)^oz of a real field */
int kgo_spectral_deriv(int N, double L, const double* u, int ox, int oy, int oz, double* out);

/* solver: lam is the coefficient of the cubic term (1 for Eq. (1)); v0 may be NULL */
kgo_state* kgo_create(int N, double L, double dt, double lam, const double* u0, const double* v0);
void kgo_destroy(kgo_state* s);
/* advance nsteps; threshold > 0 enables the blow-up check max|u^n| > threshold, which
 * freezes the state at level n, stores n in *blowup_level and returns 1 */
int kgo_step(kgo_state* s, int nsteps, double threshold, long* blowup_level);
long kgo_level(const kgo_state* s);
double kgo_last_maxabs(const kgo_state* s);
int kgo_fetch(const kgo_state* s, double* u);                            /* u^n, N^3 doubles */
int kgo_fetch_spectral(const kgo_state* s, kgo_complex* a, kgo_complex* b);  /* uh^n, uh^{n-1} */
int kgo_energy_parts(kgo_state* s, double* Q, double* Pn, double* Pnm1);
int kgo_energy(kgo_state* s, double* E);                                 /* E^{n-1/2} */

/* continuous energy at t = 0 (spectral gradient) and low-mode shell energies */
int kgo_energy_initial(int N, double L, double lam, const double* u0, const double* v0, double* E);
int kgo_shell_energies(int N, double L, const double* u0, double* out4);

/* complex field (full N^3 spectrum [kz][ky][kx], kx in FFT order; F = lam |u|^2 u;
 * every mode has weight 1 in Q; P = lam (h^3/4) sum |u|^4).  u0, v0, u: N^3 complex */
typedef struct kgoc_state kgoc_state;
int kgo_fft3d(int N, kgo_complex* a, int sign);                        /* in place, unnormalised */
kgoc_state* kgoc_create(int N, double L, double dt, double lam, const kgo_complex* u0, const kgo_complex* v0);
void kgoc_destroy(kgoc_state* s);
int kgoc_step(kgoc_state* s, int nsteps, double threshold, long* blowup_level);
long kgoc_level(const kgoc_state* s);
double kgoc_last_maxabs(const kgoc_state* s);
int kgoc_fetch(kgoc_state* s, kgo_complex* u);
int kgoc_fetch_spectral(const kgoc_state* s, kgo_complex* a, kgo_complex* b);
int kgoc_energy_parts(kgoc_state* s, double* Q, double* Pn, double* Pnm1);
int kgoc_energy(kgoc_state* s, double* E);

int kgo_num_threads(void);
void kgo_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
