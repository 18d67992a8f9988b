/*
 * pfsh.h -- C ABI of the GB300 PFASST-SH hot path.
 *
 * Method: Hamon, Schreiber & Minion, "Parallel-in-Time Multi-Level
 * Integration of the Shallow-Water Equations on the Rotating Sphere"
 * (arXiv:1904.05988).  Section numbers, equation labels and the algorithm
 * number below refer to that paper.
 *
 * General conventions
 * -------------------
 * Spectral layout.  A scalar field truncated at degree T has
 *   ncoef(T) = (T+1)(T+2)/2
 * complex coefficients xi_n^m (0 <= m <= n <= T) stored m-major:
 *   offset(m, n) = m*(2T+3-m)/2 + (n - m),
 * each as two doubles (re, im), i.e. `double[ncoef][2]`.  Coefficients with
 * m = 0 are real (their imaginary part is ignored on input, 0 on output).
 * The basis is P_n^m(mu) e^{i m lambda} with P_n^m the associated Legendre
 * function normalised to unit L2 norm on [-1, 1] without the
 * Condon-Shortley phase (Section 3, Eq. spectral_to_physical_space); a real
 * field equals sum_n xi_n^0 P_n^0 + 2 Re sum_{m>0} xi_n^m P_n^m e^{i m lambda}.
 * (The paper's ordering of Eq. spectral_space is garbled; this layout is
 * the m-major reading.)
 *
 * A shallow-water state is [Phi, zeta, delta] (Section 2): `double
 * [3][ncoef][2]`; a batch of B states is `double [B][3][ncoef][2]`.
 *
 * Grid layout.  Gaussian grid of nlat latitudes (mu_j = sin(phi_j) the roots
 * of P_nlat, north to south) by nlon equally spaced longitudes
 * lambda_k = 2 pi k / nlon: `real [batch][nlat][nlon]`, row-major.
 *
 * Memory.  Every data pointer passed to a compute call is a DEVICE pointer
 * owned by the caller; it must stay valid until the work queued on `stream`
 * has finished.  Plans, contexts, levels and PFASST objects own their tables
 * and workspaces (allocated by *_create, released by *_destroy; those two
 * synchronise the device).  Compute calls are asynchronous on `stream`
 * (NULL = legacy default stream) and never allocate.  One object may be used
 * by one stream at a time.
 *
 * Errors.  Every call returns PFSH_OK (0) or a negative pfsh_status; nothing
 * aborts the process.  Argument errors are detected on the host before any
 * work is queued.  pfsh_last_error() returns a thread-local description of
 * the last failure.  Device-side checks (non-finite values where enabled,
 * bounded waits) write a status word that pfsh_sync_status() reads.
 */
#ifndef PFSH_H
#define PFSH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* CUDA stream handle (identical to cudaStream_t). */
typedef struct CUstream_st *pfsh_stream_t;

typedef enum {
  PFSH_OK = 0,
  PFSH_EINVAL = -1,       /* invalid argument (checked on the host)          */
  PFSH_ENOMEM = -2,       /* device or host allocation failed in *_create     */
  PFSH_ECUDA = -3,        /* a CUDA runtime/driver call failed                */
  PFSH_EUNSUPPORTED = -4, /* valid request the library/device cannot serve  */
  PFSH_ETIMEOUT = -5,     /* a bounded device-side wait gave up               */
  PFSH_ENUMERIC = -6      /* device-side check found a non-finite value       */
} pfsh_status;

/* Arithmetic of the Legendre contractions (and of the FFT/grid stage).
 * PFSH_FP64: everything in float64 (the plain FP64 GPU path).
 * The others keep spectral data, recurrences, nodes/weights and all SDC/FAS
 * bookkeeping in float64 and run FFTs and grid products in float32:
 *   PFSH_FP32   Legendre in float32 on CUDA cores,
 *   PFSH_BF16   Legendre on tensor cores, bf16 operands, fp32 accumulation,
 *   PFSH_FP16   as BF16 with fp16 operands; transforms only: inputs must lie
 *               in the fp16 range (|x| < 65504, relative precision lost
 *               below 6e-5), which the right-hand side's flux products do
 *               not, so swe_ctx_create refuses FP16 plans (EUNSUPPORTED),
 *   PFSH_BF16X3 split bf16 hi/lo products (hi*hi + hi*lo + lo*hi), fp32 acc.
 *               (each operand to about 16 bits),
 *   PFSH_BF16X6 three-part bf16 split x = hi + mid + lo (about 24 bits, the
 *               precision of fp32) and the six products of the parts whose
 *               exponents sum above 2^-24, fp32 accumulation. */
typedef enum {
  PFSH_FP64 = 0,
  PFSH_FP32 = 1,
  PFSH_BF16 = 2,
  PFSH_FP16 = 3,
  PFSH_BF16X3 = 4,
  PFSH_BF16X6 = 5
} pfsh_prec;

typedef struct sht_plan sht_plan;
typedef struct swe_ctx swe_ctx;
typedef struct sdc_level sdc_level;
typedef struct pfasst pfasst;

/* ------------------------------------------------------------------------ */
/* Spherical-harmonic transform (Section 3)                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
  int T, nlat, nlon, ncoef, max_batch, prec;
  size_t device_bytes;   /* tables + workspace held by the plan             */
  const double *mu;      /* host copy of the nlat Gaussian latitudes (sin)  */
  const double *w;       /* host copy of the nlat Gauss weights             */
  int tc_tiles[2][8];    /* tensor-core forms: row tiles per order used by
                          * [0] synthesis / [1] analysis for a launch of
                          * 1..8 blocks of 128 real columns (0 otherwise)   */
} sht_info;

/* Tensor-core forms are autotuned at creation: for every launch width the
 * plan can see (blocks of 128 real columns up to 2 max_batch), the per-order
 * GEMMs are timed with their output rows in ceil(rows/256) and in twice as
 * many tiles, and the faster tiling is used for launches of that width (the
 * results are bitwise the same: tiles split output rows, not the sums).
 * Choices are cached per (T, nlat, precision, direction, width) for the
 * process and, if the environment variable PFSH_TUNE_CACHE names a file, in
 * that file (JSON lines).  PFSH_TC_TILES=1 or 2 pins the tiling instead.  */
/* Create a transform plan for truncation T on an nlat x nlon Gaussian grid.
 * Requires T >= 1, nlat even, nlat >= T+2, nlon > 2(T+1), nlon even with all
 * prime factors <= 61, and 1 <= max_batch.  `max_batch` bounds the number of
 * fields (sht_*) per internal pass; larger batches are processed in chunks.
 * Builds Gaussian nodes/weights and the associated Legendre table by an FP64
 * recurrence on the device.  Synchronises the device. */
int sht_plan_create(sht_plan **out, int T, int nlat, int nlon, int max_batch,
                    int prec);
int sht_plan_destroy(sht_plan *plan);
int sht_plan_query(const sht_plan *plan, sht_info *info);

/* Synthesis (Eq. spectral_to_physical_space): spec [batch][ncoef(T)][2]
 * (double) -> grid [batch][nlat][nlon] (double for PFSH_FP64 plans, float
 * otherwise).  `spec` and `grid` must not overlap. */
int sht_inverse(sht_plan *plan, const double *spec, void *grid, int batch,
                pfsh_stream_t stream);

/* Analysis (DFT in longitude, then Gauss-Legendre quadrature in latitude):
 * grid [batch][nlat][nlon] -> spec [batch][ncoef(T)][2]. */
int sht_forward(sht_plan *plan, const void *grid, double *spec, int batch,
                pfsh_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Shallow-water right-hand sides and implicit solve (Sections 2, 4, 5.4)   */
/* ------------------------------------------------------------------------ */

/* Where the Coriolis force goes in the IMEX split (Section 4):
 * EXPLICIT (the paper's split): f = 2 omega mu enters N through
 *   eta = zeta + f, and F_I = L is diagonal in (n, m).
 * IMPLICIT: the linear Coriolis tendency C = [0, -div(f V), curl(f V)]
 *   moves to F_I = L + C and N is evaluated with eta = zeta (F_E + F_I is
 *   unchanged).  C couples degree n to n +- 1 within an order m, so the
 *   implicit system of an order is banded (two tridiagonal chains). */
#define PFSH_CORIOLIS_EXPLICIT 0
#define PFSH_CORIOLIS_IMPLICIT 1

typedef struct {
  double a;      /* sphere radius [m]                                        */
  double omega;  /* rotation rate [1/s]; f = 2 omega mu                      */
  double nu;     /* second-order diffusion coefficient [m^2/s]               */
  double phibar; /* mean geopotential Phibar = g hbar [m^2/s^2]              */
  int coriolis;  /* PFSH_CORIOLIS_EXPLICIT (0) or PFSH_CORIOLIS_IMPLICIT     */
  int implicit_split; /* SDC node solve (Section 5.1.1): 0 = one solve of
                 * x - h F_I(x) = b; 1 = two substeps, the physical linear
                 * terms (gravity waves, plus Coriolis when implicit) with the
                 * diffusion of the previous iterate, then the diffusion:
                 *   x* - h L0(x*) = b + h D(old),  x - h D(x) = x* - h D(old)
                 * (D = the diffusion part of F_I; each substep carries its
                 * own correction term, so converged sweeps reach the same
                 * collocation solution).  swe_implicit_solve always solves
                 * x - h F_I(x) = b in one step.                              */
} swe_params;

/* The context keeps a reference to `plan` (which must outlive it) and owns
 * the RHS workspace for up to plan->max_batch/4 states per pass. */
int swe_ctx_create(swe_ctx **out, sht_plan *plan, const swe_params *params);
int swe_ctx_destroy(swe_ctx *ctx);

/* F_E = N(Theta) (Eq. nonlinear_operators, evaluated by the spectral
 * transform method) and F_I = L(Theta) (Eq. linear_wave_motion_induced_by_
 * gravitational_forces) for B states [B][3][ncoef][2]; with
 * PFSH_CORIOLIS_IMPLICIT, F_E = N with eta = zeta and F_I = L + C.  fE is
 * required, fI may be NULL.  Outputs must not overlap `state`. */
int swe_rhs(swe_ctx *ctx, const double *state, double *fE, double *fI, int B,
            pfsh_stream_t stream);

/* Solve x - h F_I(x) = b (Eq. implicit_systems): coefficient by coefficient
 * for PFSH_CORIOLIS_EXPLICIT; with PFSH_CORIOLIS_IMPLICIT, one banded solve
 * per order m (FP64 elimination along n, no pivoting: stable because the
 * Coriolis coupling is skew-Hermitian in the energy weights).  b, x
 * [B][3][ncoef][2]; x may alias b.  Calls on one context must not run
 * concurrently on different streams (they share a factor table). */
int swe_implicit_solve(swe_ctx *ctx, const double *b, double *x, double h,
                       int B, pfsh_stream_t stream);

/* ------------------------------------------------------------------------ */
/* IMEX-SDC on Gauss-Lobatto nodes (Section 5.1.1)                           */
/* ------------------------------------------------------------------------ */

/* A level: SWE context, num_nodes Gauss-Lobatto nodes in [t, t+dt] (2..9),
 * and workspace for up to max_batch states. */
int sdc_level_create(sdc_level **out, swe_ctx *ctx, int num_nodes, double dt,
                     int max_batch);
int sdc_level_destroy(sdc_level *level);

/* Initial iterate: copy theta0 [B][3][ncoef][2] to every node and fill the
 * right-hand sides at every node with F(theta0).  theta, fE, fI:
 * [num_nodes][B][3][ncoef][2]. */
int sdc_spread(sdc_level *level, const double *theta0, double *theta,
               double *fE, double *fI, int B, pfsh_stream_t stream);

/* One sweep of Eq. update_equation_sdcq_discrete_form (with the FAS term
 * tau of Eq. modified_update_equation_sdcq_discrete_form when tau != NULL,
 * tau [num_nodes][B][3][ncoef][2], cumulative from the left end): updates
 * theta, fE, fI at nodes 1..M in place.  Node 0 holds the initial value and
 * its right-hand sides must be current. */
int sdc_sweep(sdc_level *level, double *theta, double *fE, double *fI,
              const double *tau, int B, pfsh_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Two-level PFASST, all time slices on one GPU (Sections 5.1.2-5.3, Alg. 1) */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n_ts;                   /* time slices solved together               */
  int fine_nodes, coarse_nodes; /* Gauss-Lobatto nodes per level (2, 3, 5) */
  int Tf, nlat_f, nlon_f;     /* fine truncation and grid                 */
  int Tc, nlat_c, nlon_c;     /* coarse truncation (Tc <= Tf) and grid    */
  double dt;                  /* time-step size of every slice [s]         */
  swe_params phys;
  int prec;                   /* pfsh_prec of both levels' transforms      */
  int slice_groups;           /* pipeline depth of an iteration: slices are
                               * split into this many groups of consecutive
                               * slices, and the coarse chain (Step C) of a
                               * group overlaps Steps A/B of the next ones.
                               * 0 = automatic (1 for FP64, 2 otherwise);
                               * clamped so that every group holds >= 4
                               * slices.  Results do not depend on it.     */
} pfasst_config;

/* Allocates every slice's fine and coarse space-time arrays. */
int pfasst_create(pfasst **out, const pfasst_config *cfg);
int pfasst_destroy(pfasst *pf);

/* Initial value of the first slice: theta0 [3][ncoef(Tf)][2] (device). */
int pfasst_set_initial(pfasst *pf, const double *theta0, pfsh_stream_t stream);

/* Prediction step (Section 5.2.1): broadcast, restrict, n_ts rounds of coarse
 * sweeps (slice n sweeps n+1 times), interpolate, evaluate fine F. */
int pfasst_predict(pfasst *pf, pfsh_stream_t stream);

/* One PFASST iteration (Algorithm 1) over all slices.  last != 0 performs
 * Step A only (the paper's last iteration).  Work is issued on `stream` and
 * on an internal stream that joins back into `stream` before the call's
 * work is complete, so stream order for the caller is unchanged. */
int pfasst_iteration(pfasst *pf, int last, pfsh_stream_t stream);

/* `count` consecutive PFASST iterations (Algorithm 1), the last of them Step A
 * only when last != 0; the same results as `count` calls of pfasst_iteration.
 * Within the block the slice groups form a wavefront across iterations: the
 * fine sweep of group g in iteration k+1 starts as soon as the coarse chain
 * of group g in iteration k has finished, beside the chain of the later
 * groups.  Stream semantics as pfasst_iteration.  EINVAL if count < 1. */
int pfasst_iterations(pfasst *pf, int count, int last, pfsh_stream_t stream);

/* Ensembles of independent instances (uneven batches: members may differ in
 * truncation, grid, nodes, slices and precision).  Every member is a full
 * pfasst object (pfasst_ensemble_member returns it, e.g. for
 * pfasst_set_initial and pfasst_get); predictor and iteration blocks of all
 * members run concurrently, each member on its own stream pair, the
 * iteration blocks captured into one CUDA graph per (count, last).  Results
 * are those of the members run one by one.  The ensemble owns its members. */
typedef struct pfasst_ensemble pfasst_ensemble;
int pfasst_ensemble_create(pfasst_ensemble **out, const pfasst_config *cfgs, int n);
int pfasst_ensemble_destroy(pfasst_ensemble *e);
/* NULL (and pfsh_last_error set) if i is out of range. */
pfasst *pfasst_ensemble_member(pfasst_ensemble *e, int i);
int pfasst_ensemble_predict(pfasst_ensemble *e, pfsh_stream_t stream);
int pfasst_ensemble_iterations(pfasst_ensemble *e, int count, int last, pfsh_stream_t stream);

/* Residual check for a variable number of iterations: res[n] (device,
 * n_ts doubles) = max over the coefficients of slice n of |theta_f(end) -
 * theta_f(end) at the previous call| / max |theta_f(end)| (fine level, last
 * node), and the current end values become the previous ones.  Call it once
 * after the predictor, then after every iteration (or block) and stop when
 * max_n res[n] is below a tolerance.  Stream-ordered; no host sync. */
int pfasst_residual(pfasst *pf, double *res, pfsh_stream_t stream);

/* Copy one node of one slice to `out` (device, [3][ncoef][2]); level 0 =
 * fine, 1 = coarse. */
int pfasst_get(pfasst *pf, int level, int slice, int node, double *out,
               pfsh_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Synthesis without any device allocation (no counterpart in the paper)     */
/* ------------------------------------------------------------------------ */

/* FP64 synthesis (same result as sht_inverse on an FP64 plan) for callers
 * that may not allocate device memory: for example a loop running under a
 * no-allocation policy after start-up, or an application whose memory pool
 * owns every device byte, and which therefore cannot create an sht_plan
 * (plans get their tables and workspace from cudaMalloc).  Only the caller's
 * spec [batch][ncoef(T)][2] (device, input) and grid [batch][nlat][nlon]
 * (device, double, output) are used; nothing is allocated.  The Legendre
 * functions are evaluated on the fly; Gaussian latitudes, twiddles and the
 * intermediate Fourier coefficients live in a fixed 4 MiB device array
 * inside this library, which every GPU that loads the library keeps until
 * the process exits.
 * Limits: 1 <= T <= 127, nlat even >= T+2, nlon even > 2(T+1) with prime
 * factors <= 61 and 2*(nlon + nlon/16 + 1)*16 bytes <= 227 KiB (the
 * longitude transform keeps two padded rows in shared memory, so nlon up to
 * about 6800), and (T+1)*nlat*batch*16 bytes plus the latitudes
 * (nlat*8 bytes) and FFT twiddles (at most 3*nlon*16 bytes), each rounded up
 * to 256, within 4 MiB; larger requests return PFSH_EINVAL before any work
 * is queued (split the batch).
 * The first call on a device looks up the device address of that array
 * (cudaGetSymbolAddress) and remembers it; make that first call before any
 * stream capture.  The call launches on the current device: spec and grid
 * must live there.  All calls share the one array and every call rewrites
 * what it reads, so no state carries over between calls; calls whose work
 * overlaps on the GPU (different streams, no ordering) race on it.
 * Asynchronous on `stream` like the other compute calls. */
int sht_inverse_noalloc(int T, int nlat, int nlon, const double *spec,
                        double *grid, int batch, pfsh_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Status                                                                    */
/* ------------------------------------------------------------------------ */

/* Synchronise `stream` and report the sticky device-side status of all
 * objects of this library (PFSH_OK, PFSH_ETIMEOUT, PFSH_ENUMERIC) and any
 * CUDA error; clears the status word. */
int pfsh_sync_status(pfsh_stream_t stream);

/* Thread-local, NUL-terminated description of the last failure ("" if none). */
const char *pfsh_last_error(void);

/* on != 0: from now on swe_rhs (F_E, F_I), sdc_sweep (every node of theta),
 * pfasst_predict, pfasst_iteration and pfasst_iterations (the fine end value
 * of every slice) append one kernel that scans their results and records a
 * non-finite component (NaN, +-Inf) in the status word, so that the next
 * pfsh_sync_status returns PFSH_ENUMERIC.  Off by default (it costs one read
 * of the results).  Process-wide; the check runs outside the CUDA graphs of
 * the PFASST calls. */
int pfsh_set_check_finite(int on);

/* Self-test of the bounded device-side waits (no counterpart in the paper):
 * one CTA allocates tensor memory, waits on an mbarrier that nothing arms
 * with the poll limit `polls` (1..2^20) of the library's bounded wait, frees
 * its tensor memory and returns; the status word then holds the timeout, so
 * the next pfsh_sync_status returns PFSH_ETIMEOUT and the context stays
 * usable.  Asynchronous on `stream`. */
int pfsh_selftest_wait(unsigned polls, pfsh_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Diagnostics (no counterpart in the paper)                                 */
/* ------------------------------------------------------------------------ */

/* Number of CUDA kernels this library has launched in this process. */
unsigned long long pfsh_kernel_launches(void);

/* on != 0: from now on record a CUDA event pair on the launching stream
 * around every kernel launch (adds a little host overhead per launch);
 * on == 0: stop recording.  Enabling clears previous records. */
int pfsh_profiler_enable(int on);

/* Measured FMA throughput of the FP64 (prec = PFSH_FP64) or FP32
 * (PFSH_FP32) pipe of the current device in TFLOP/s (FMA = 2 flops): a loop
 * of independent FMA chains on every SM, timed with CUDA events, best of 5
 * launches.  The roofline denominator of kernels bound by that pipe.
 * Synchronises its own stream; takes well under a second. */
int pfsh_alu_peak(int prec, double *tflops);

/* Synchronise the device and write a JSON object
 * {"<kernel>": [launches, total_ms], ...} of the records so far into buf
 * (NUL-terminated, truncated to n bytes).  Returns the length needed. */
int pfsh_profiler_report(char *buf, size_t n);

#ifdef __cplusplus
}
#endif

#endif /* PFSH_H */
