/*
 * kg.h -- C ABI of libkg.so, a GB300 (sm_103a) stepper for the real cubic
 * Klein-Gordon equation on a periodic cube,
 *
 *     u_tt - Laplace(u) + u = |u|^2 u,                  Aseeri et al., Eq. (1),
 *
 * advanced with the second-order semi-implicit scheme of section 1.1.2, Eq. (2),
 * in Fourier space, the cubic term formed in real space: every step is one
 * complex-to-real 3D FFT, the pointwise cube, one real-to-complex 3D FFT and the
 * per-mode update (section 1.1.2, "two FFTs per time step").
 *
 * Conventions shared by every entry point
 *   grid      N^3 points on [-L/2, L/2)^3, x_j = -L/2 + j L/N, N in {16,32,...,512}.
 *             Physical arrays are N^3 doubles, [z][y][x] with x fastest.
 *   spectrum  unnormalised forward DFT, half spectrum kx = 0..N/2; Fourier state
 *             uh^n, uh^{n-1} kept in FP64 on the device.  The C2R inverse keeps the
 *             real parts of the kx = 0 and kx = N/2 entries; no dealiasing; the
 *             Nyquist wavenumber keeps k^2 = (pi N / L)^2.
 *   update    uh^{n+1} = 2 c_k uh^n - uh^{n-1} + 2 beta_k F^n_k with
 *             omega_k^2 = 1 + k^2, c_k = (1 - dt^2 omega^2/4)/(1 + dt^2 omega^2/4),
 *             beta_k = (dt^2/2)/(1 + dt^2 omega^2/4), F = lam u^3 (lam = 1: Eq. (1)).
 *   startup   the paper gives none: uh^{-1} = c_k uh^0 - dt vh^0 + beta_k F^0_k
 *             (the symmetric level (u^1 - u^{-1})/(2 dt) = v0 put into Eq. (2)).
 *   energy    the paper gives the continuous functional of section 1.1; the
 *             discrete one here is E^{n-1/2} = Q^{n-1/2} - (P^{n-1} + P^n)/2 with
 *             Q^{n+1/2} = (h^3/N^3) sum_k w_k [ |(uh^{n+1}-uh^n)/dt|^2/2
 *                                          + omega_k^2 |(uh^{n+1}+uh^n)/2|^2/2 ],
 *             P^n = lam (h^3/4) sum_x (u^n)^4, w_k = 1 on kx = 0, N/2 and 2 elsewhere.
 *
 * Context and threading: one global context per process, not thread-safe.  Calls
 * are ordered on one CUDA stream (the library's own, or the caller's via
 * kg_set_stream).  Every entry point returns KG_OK (0) or a negative status;
 * kg_last_error() then describes the failure.  No C++ exception crosses the ABI.
 * Host pointers are only read (or written) during the call; the library keeps no
 * reference to caller memory.
 */
#ifndef KG_H
#define KG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define KG_OK 0
#define KG_EINVAL (-1)    /* bad argument: NULL pointer, non-finite input, dt <= 0, ... */
#define KG_ENOTSUP (-2)   /* N outside the supported set, or a combination this build lacks */
#define KG_ENOMEM (-3)    /* device or host allocation failed; nothing is leaked */
#define KG_ECUDA (-4)     /* a CUDA runtime call failed; see kg_last_error() */
#define KG_ETIMEOUT (-5)  /* a bounded device-side wait gave up */
#define KG_EDRIFT (-6)    /* energy watchdog: |E - E_0| > drift_tol |E_0| */
#define KG_ENOTIMPL (-7)  /* entry point not available in this build */
#define KG_ESTATE (-8)    /* call out of order (e.g. kg_step before kg_init) */

/* arithmetic of the FFT passes (the state uh, the update and the sums are FP64 in all).
 * The set-up transforms of kg_init / kg_init_complex and the read-out of kg_fetch /
 * kg_fetch_complex run in double-float for KG_DF64 and in IEEE FP64 for the other two. */
#define KG_FP64 0   /* IEEE FP64 everywhere */
#define KG_DF64 1   /* FFT and cube in double-float (pairs of FP32, ~48-bit significand) */
#define KG_MIXED 2  /* FFT and cube in FP32 (section 1.1.2 scheme, FP32/FP64 split) */

typedef struct kg_options {
    int precision;          /* KG_FP64, KG_DF64 (default) or KG_MIXED; takes effect at kg_init */
    int energy_every;       /* record Q and P during kg_step every this many levels (0: never) */
    double nonlinearity;    /* lam, coefficient of u^3 (default 1.0 = Eq. (1); 0 = linear) */
    double blowup_threshold;/* > 0: freeze the state once max|u^n| exceeds it (default 0: off) */
    double drift_tol;       /* > 0: kg_energy returns KG_EDRIFT past this relative drift */
    const char* tune_cache; /* batched ensemble: the autotuner's cache file, as kg_ens_set_tune_cache
                             * (copied by kg_set_options; NULL leaves the current file, "" sets none;
                             * kg_get_options returns the library's copy or NULL) */
} kg_options;

/* Set up the solver: N^3 grid of side L, time step dt, initial field u0 and
 * velocity v0 (host pointers, N^3 doubles each, [z][y][x]; v0 may be NULL = 0).
 * Both are copied; the caller keeps ownership.  Replaces any previous context.
 * Level after the call: n = 0.  Errors: KG_EINVAL, KG_ENOTSUP, KG_ENOMEM, KG_ECUDA. */
int kg_init(int N, double L, double dt, const double* u0, const double* v0);

/* As kg_init with device pointers (N^3 doubles each, v0 may be NULL). */
int kg_init_device(int N, double L, double dt, const double* d_u0, const double* d_v0);

/* Enqueue n steps of Eq. (2) on the context's stream; returns once enqueued.
 * Errors: KG_ESTATE (no context), KG_EINVAL (n < 0), KG_ECUDA. */
int kg_step(int n);

/* Synchronise and write E^{n-1/2} at the current level n (definition above).
 * Returns KG_EDRIFT (with *E written) when the drift watchdog trips.  P^n needs u^n, which
 * only the next step's x pass forms: for a real field stepped by separate passes this call
 * runs that x pass now (its blow-up check of u^n included, so a blow-up at level n shows in
 * kg_status from here on) and the next kg_step / kg_step_timed skips it, so an energy
 * evaluation costs no extra pass; otherwise (complex field, fused xy form, frozen state) a
 * read-only pass or the FP64 state supplies P^n.  A second call at the same level returns
 * the same value. */
int kg_energy(double* E);

/* Synchronise and write u^n (N^3 doubles, [z][y][x]) into caller-owned host memory. */
int kg_fetch(double* u);

/* Same into caller-owned device memory (N^3 doubles); enqueued, no host sync. */
int kg_fetch_device(double* d_u);

/* Release the context and all device memory.  Safe to call twice. */
int kg_finalize(void);

/* Use this CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * for all later work; NULL returns to the library's own stream. */
int kg_set_stream(void* stream);

int kg_set_options(const kg_options* opt);  /* copies *opt; precision applies at the next init */
int kg_get_options(kg_options* opt);

/* ---- time-stepping scheme (section 3 names higher-order time stepping as future work
 * and gives no scheme; the fourth-order one here is an outside specification) ----
 * KG_SCHEME_EQ2 (default): Eq. (2).
 * KG_SCHEME_COMPOSED4: Eq. (2) written as the equivalent one-step kick-drift-kick map on
 * (uh, velocity) -- per mode p += (h/2) G_h(uh), uh += h p, p += (h/2) G_h(uh), with
 * G_h = (F - omega^2 uh) / (1 + omega^2 h^2/4), which with h = dt is exactly Eq. (2) and its
 * startup level -- composed as Yoshida's triple jump (Phys. Lett. A 150 (1990) 262): a step
 * of length dt is three substeps of lengths g1 dt, g2 dt, g1 dt, g1 = 1/(2 - 2^{1/3}),
 * g2 = 1 - 2 g1.  Fourth order in dt; one step costs three evaluations of F (three passes
 * of the step's kernels; adjacent half kicks are merged).  kg_step(n) advances n steps and
 * kg_status reports steps; the blow-up check and the max |u| of kg_status look at the
 * field at integer steps only.  Real fields only (kg_init_complex: KG_ENOTSUP);
 * energy_every and drift_tol must be 0 (kg_init: KG_EINVAL).  kg_energy returns the
 * continuous energy of section 1.1 at step n, evaluated in FP64 with the synchronised
 * velocity p^n: (h^3/N^3) sum_k w_k (|p^n_k|^2 + omega_k^2 |uh^n_k|^2)/2 - lam (h^3/4) sum u^4
 * (the composition conserves it to O(dt^4)).  kg_fetch_spectral returns (uh^n, P^n) where the stored velocity variable is
 * P^n = p^n - (g1 dt/2) G_{g1 dt}(uh^n).  The scheme takes effect at the next kg_init (or
 * comes from the checkpoint in kg_load_state). */
#define KG_SCHEME_EQ2 0
#define KG_SCHEME_COMPOSED4 1
int kg_set_scheme(int scheme);   /* KG_EINVAL for an unknown scheme */
int kg_get_scheme(int* scheme);  /* the scheme the next kg_init uses */

/* ---- xy-plane fusion (FP32 passes) ----
 * The transforms of a step that mix values within one z-plane only -- the inverse y
 * transforms that end a step, the x pass (C2R, cube, R2C; section 1.1.2) and the forward
 * y transforms that begin the next -- run as one kernel in which a cluster of 8 CTAs holds
 * a whole plane of the FP32 work array in its distributed shared memory, so the plane is
 * read and written once instead of three times (the paper's section 2.1 counts these
 * passes over memory as the cost of the FFT).  on = 1 selects it for contexts that can
 * use it: KG_MIXED, a real field, KG_SCHEME_EQ2, N >= 64; other contexts ignore it.  The
 * arithmetic is that of the separate passes, so the results are identical to them
 * (up to the summation order of the recorded sum of u^4).  Takes effect at the next
 * kg_step; between kg_step calls the state is the same in both forms.  Default 0.
 * kg_get_xy_fusion: *on as set; *active (may be NULL) = 1 if the current context uses it. */
int kg_set_xy_fusion(int on);    /* KG_EINVAL unless on is 0 or 1 */
int kg_get_xy_fusion(int* on, int* active);

/* Current level n, blow-up state (1 if frozen, with the level it froze at) and the
 * max |u| seen by the last step (that of u^{n-1}).  Synchronises. */
int kg_status(long long* level, int* frozen, long long* blowup_level, double* maxabs);

/* Copy the Fourier state uh^n and uh^{n-1} (N*N*(N/2+1) complex doubles each,
 * interleaved re/im, [kz][ky][kx]) to host memory; either pointer may be NULL. */
int kg_fetch_spectral(double* a, double* b);

/* Instrumentation: enqueue n steps launching each kernel separately, timing them
 * with CUDA events on the context's stream; ms[0..5] receive the summed device time
 * of the x pass (with its finaliser), forward y, the z pass, its update part, its
 * inverse-z part and inverse y.  The z pass (forward z FFT, update, inverse z FFT) is
 * one kernel, so ms[2] holds all of it with its finaliser and ms[3], ms[4] receive 0.
 * Synchronises. */
int kg_step_timed(int n, float* ms);

/* Bytes of device memory the context holds. */
int kg_memory(size_t* bytes);

/* ---- complex field (section 1.1.2: the paper's implementation allows a complex u) ----
 * The same scheme for complex u with the nonlinearity lam |u|^2 u (Eq. (1) as printed):
 * the spectrum is the full N^3 array [kz][ky][kx] with kx = 0..N-1 in FFT order (no
 * Hermitian symmetry, no C2R rule), every mode has weight 1 in Q, P^n = lam (h^3/4)
 * sum |u^n|^4, and the blow-up check and kg_status use max |u^n| = max sqrt(re^2 + im^2).
 * kg_step, kg_energy, kg_status, kg_fetch_spectral (N^3 complex values each),
 * kg_step_timed, kg_save_state and kg_load_state work on either kind of context;
 * kg_fetch / kg_fetch_device refuse a complex one (KG_ESTATE) and the calls below
 * refuse a real one. */

/* As kg_init for a complex field: u0, v0 (v0 may be NULL) are host pointers to N^3
 * complex values, interleaved re/im (2 N^3 doubles), [z][y][x] with x fastest. */
int kg_init_complex(int N, double L, double dt, const double* u0, const double* v0);

/* As kg_init_complex with device pointers. */
int kg_init_complex_device(int N, double L, double dt, const double* d_u0, const double* d_v0);

/* Synchronise and write the complex u^n (2 N^3 doubles, interleaved) to host memory. */
int kg_fetch_complex(double* u);

/* Same into caller-owned device memory (2 N^3 doubles); enqueued, no host sync. */
int kg_fetch_complex_device(double* d_u);

/* ---- checkpoint / resume (the paper has no counterpart; long blow-up runs need it) ----
 * A checkpoint is one host byte buffer: a kg_state_header followed by the payload,
 * uh^n then uh^{n-1} (N*N*(N/2+1) complex doubles each, interleaved re/im,
 * [kz][ky][kx]), in the byte order of the machine that wrote it (little-endian on
 * both x86-64 and Arm64).  Only the FP64 state is stored: the work array is
 * rebuilt from uh^n on load by the same inverse transforms a step ends with, so a
 * resumed run continues bit for bit as the uninterrupted one would. */
#define KG_STATE_MAGIC "KGSTATE1"
#define KG_STATE_VERSION 1u

typedef struct kg_state_header {
    char magic[8];               /* KG_STATE_MAGIC, no terminating NUL */
    unsigned int version;        /* KG_STATE_VERSION */
    unsigned int header_bytes;   /* sizeof(kg_state_header) = 256 */
    int N, precision, energy_every, frozen;
    double L, dt, nonlinearity, blowup_threshold, drift_tol;
    long long level;             /* n of uh^n */
    long long blowup_level;      /* -1 unless frozen */
    double maxabs_last;          /* max |u| seen by the last step */
    double P_last;               /* last recorded P and Q with their levels */
    long long P_last_level;
    double Q_last;
    long long Q_last_level;
    int have_E0, pad0;
    double E0;                   /* the drift watchdog's first energy */
    unsigned long long payload_bytes;   /* 2 * 16 * N*N*(N/2+1) (complex field: 2 * 16 * N^3) */
    unsigned long long checksum;        /* kg_state_checksum of the payload */
    int complex_field;                  /* 1: complex field (payload 2 * 16 * N^3 bytes) */
    int scheme;                         /* KG_SCHEME_EQ2 or KG_SCHEME_COMPOSED4 */
    unsigned char reserved[256 - 168];  /* zero */
} kg_state_header;

/* Write the current context into h (cap bytes).  *used receives the checkpoint
 * size in every case; h == NULL only asks for that size.  Synchronises.
 * Errors: KG_ESTATE (no context), KG_EINVAL (used NULL, or cap too small: nothing
 * written), KG_ECUDA. */
int kg_save_state(void* h, size_t cap, size_t* used);

/* Replace the context by the checkpoint in h (len bytes): the run's grid, time
 * step, scheme and options (precision, energy_every, nonlinearity, blowup_threshold,
 * drift_tol) become the current ones, as kg_init plus kg_set_options and
 * kg_set_scheme would make them, and the level, blow-up state and recorded energies are restored.  The
 * header and the payload checksum are checked before anything is replaced.
 * Errors: KG_EINVAL (bad magic, version, size, field or checksum) and KG_ENOTSUP
 * keep the old context and options; after KG_ENOMEM or KG_ECUDA no context remains
 * and the options are the checkpoint's. */
int kg_load_state(const void* h, size_t len);

/* 64-bit checksum of a checkpoint payload: the sum, modulo 2^64, of each 8-byte
 * word rotated left by (its index mod 64), the words read in machine byte order.
 * n must be a multiple of 8. */
unsigned long long kg_state_checksum(const void* p, size_t n);

/* ---- batched parametric ensemble (blow-up studies, section 1 of the paper) ----
 * count independent instances (1..1024) on grids Ns[i] in {64, 128}, side L, step dt,
 * u0 = A[i] exp(-|x|^2 / s[i]^2), v0 = 0, in the precision and nonlinearity of the
 * current options.  Each time step of the whole ensemble is one persistent
 * cooperative kernel launch (four passes separated by bounded grid barriers), and
 * runs of steps are replayed from a captured CUDA graph.  One ensemble per process;
 * independent of the kg_init context.  Errors: KG_EINVAL, KG_ENOTSUP, KG_ENOMEM,
 * KG_ECUDA, KG_ETIMEOUT (a grid barrier wait gave up; the ensemble state is then
 * undefined and must be re-initialised). */
int kg_ens_init(int count, const int* Ns, double L, double dt, const double* A, const double* s);

/* Advance every instance that has not blown up by up to max_steps steps.  With
 * threshold > 0 an instance whose max|u^n| exceeds it is frozen at level n (its
 * blow-up level); the run ends early once all instances are frozen.  *steps_done
 * receives the number of ensemble steps launched and *ms their device time (either
 * pointer may be NULL).  Synchronises. */
int kg_ens_run(int max_steps, double threshold, long long* steps_done, double* ms);

/* Per-instance results (arrays of count entries, any may be NULL): frozen flag,
 * blow-up level (-1 if none), current level, max|u| seen by its last step. */
int kg_ens_results(int* frozen, long long* blowup_level, long long* level, double* maxabs);

/* Low-mode shell energies of uh^0, count x 4 doubles: (h^3/N^3) sum w_k omega_k^2 |uh_k|^2 / 2
 * over integer wavenumber norms |m| in {0}, (0,1], (1,2], (2,4]. */
int kg_ens_features(double* shells);

/* u^n of instance i (N^3 doubles, host memory). */
int kg_ens_fetch(int i, double* u);

/* Time every launch shape for `steps` steps on the current ensemble, keep the fastest,
 * and remember it for later kg_ens_init calls with the same precision and grid mix (and,
 * with kg_ens_set_tune_cache, in the cache file).  A shape is a schedule -- bit 0: column
 * tiles of half the default width; bit 1: the short radix stage first in transforms whose
 * length is not a power of 8 (the 128^3 instances) -- times the unit order (0: instance
 * order, 1: larger grids first) times the resident CTAs per SM.  Every shape computes the
 * same step; schedules with bit 1 differ from the others in the rounding of the
 * transforms only.  Advances the ensemble.  blocks_per_sm and order may be NULL. */
int kg_ens_tune(int steps, int* blocks_per_sm, int* order);

/* The launch shape of the current ensemble (any pointer may be NULL). */
int kg_ens_schedule(int* sched, int* blocks_per_sm, int* order);

/* Force a launch shape: sched 0..3, blocks_per_sm >= 1 (capped at what fits), order 0 or
 * 1.  KG_EINVAL otherwise, KG_ESTATE without an ensemble. */
int kg_ens_set_schedule(int sched, int blocks_per_sm, int order);

/* Text file in which kg_ens_tune stores its choice, keyed by precision, grid mix, device
 * name and SM count (one line per key, rewritten through a temporary file), and from which
 * kg_ens_init takes the shape when this process has not tuned that key.  NULL or "": no
 * file (default).  The same setting as kg_options.tune_cache. */
int kg_ens_set_tune_cache(const char* path);

int kg_ens_finalize(void);

/* The same four shell energies for count sampled Gaussians A[i] exp(-|x|^2/s[i]^2) on an
 * N^3 grid of side L (N even), without building instances (the field is separable, so its
 * low modes are products of 1D DFT sums).  shells: count x 4 doubles. */
int kg_gaussian_features(int count, int N, double L, const double* A, const double* s, double* shells);

/* ---- blow-up ranker network ----
 * The paper motivates parametric blow-up studies (section 1) but has no learned
 * component; this network is the project's: 6 inputs (A, s and four low-mode shell
 * energies, normalised by the caller) -> 128 -> 128 -> 2 with ReLU; z0 is the
 * blow-up logit, z1 the predicted log blow-up time.  Loss (mean over the batch):
 * BCE(z0, y) + y (z1 - l)^2 + (1 - y) max(log T - z1, 0)^2.  BF16 operands on the
 * tensor cores with FP32 accumulation; Adam (b1 0.9, b2 0.999, eps 1e-8) on FP32
 * master weights.  Parameters are one float vector in the order W1 (6 x 128,
 * row-major [in][out]), b1 (128), W2 (128 x 128), b2, W3 (128 x 2), b3 (2).
 * All arrays are host memory; X is n x 6 row-major. */
typedef struct kg_mlp_cfg {
    int epochs;               /* passes over the data */
    int batch;                /* rows per Adam step (a trailing partial batch is dropped) */
    double lr;                /* Adam step size */
    double T;                 /* censoring time of runs without blow-up */
    unsigned long long seed;  /* shuffling stream */
} kg_mlp_cfg;

int kg_mlp_param_count(void);                       /* length of the parameter vector */
int kg_mlp_set_params(const float* params);         /* also resets Adam's moments and step count */
int kg_mlp_get_params(float* params);
/* gradient of the mean loss over the n rows (and the loss) at the current parameters */
int kg_mlp_grad(const float* X, const float* y, const float* logt, int n, double T, float* grad, double* loss);
/* one Adam step with a caller-supplied gradient */
int kg_mlp_adam_step(const float* grad, double lr);
/* epochs of shuffled mini-batch Adam; *final_loss = mean loss of the last epoch */
int kg_mlp_train(const float* X, const float* y, const float* logt, int n, const kg_mlp_cfg* cfg, double* final_loss);
/* p_blowup = sigmoid(z0), logt = z1 (either may be NULL) */
int kg_mlp_predict(const float* X, int n, float* p_blowup, float* logt);
int kg_mlp_finalize(void);

/* Quadratic energy Q of a caller-held Fourier state pair, without allocating.
 * The paper has no counterpart: this is a service for callers that cannot call
 * cudaMalloc, such as applications whose device memory belongs to another
 * allocator or to a pool fixed at start-up, and loops that cannot take the device
 * synchronisation of cudaMalloc/cudaFree.
 *   d_cur, d_old  device arrays of N*N*(N/2+1) complex doubles (interleaved re/im,
 *                 [kz][ky][kx]) holding uh^n and uh^{n-1}; read only
 *   d_Q           device double that receives Q^{n-1/2} as defined above
 *                 (the energy of the state pair when lam = 0)
 *   stream        cudaStream_t to enqueue on (NULL: the legacy default stream)
 * Needs no context.  The partial sums go to a static device array of 8192 doubles
 * (64 KiB, held by every GPU that loads the library until the process exits),
 * which bounds the size: N must be even with N*N*(N/2+1) <= 8192*16384 modes
 * (N <= 644); larger or odd N returns KG_ENOTSUP.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current, and keeps it for the rest of the process; make that first call before any
 * stream capture.  A cudaDeviceReset on that device discards the array with the rest
 * of the device's state, and with it the kept address: do not call this entry point
 * on a device after resetting it.  All calls on a device share the array, so calls
 * that overlap on the GPU (concurrent streams) race.
 * Enqueued asynchronously; allocates nothing.  Errors: KG_ENOTSUP, KG_EINVAL
 * (NULL pointer, L or dt not finite and > 0), KG_ECUDA. */
int kg_energy_q_noalloc(int N, double L, double dt, const double* d_cur, const double* d_old, double* d_Q,
                        void* stream);

/* Description of the last failure in this thread ("" if none). */
const char* kg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KG_H */
