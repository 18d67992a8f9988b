// Internal declarations of the PFASST-SH CUDA library (not part of the ABI).
#pragma once

#include <utility>

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/pfsh.h"

namespace pfsh {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define PFSH_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ::pfsh::cuda_fail(e_, #call); \
  } while (0)

#define PFSH_CHECK_LAUNCH(what)                                     \
  do {                                                              \
    cudaError_t e_ = cudaGetLastError();                            \
    if (e_ != cudaSuccess) return ::pfsh::cuda_fail(e_, what);      \
  } while (0)

// Brackets one kernel launch: counts it and, when the profiler is on,
// records an event pair on the launching stream.
struct LaunchScope {
  LaunchScope(const char *name, cudaStream_t s);
  ~LaunchScope();
  const char *name;
  cudaStream_t stream;
  int slot;
};
#define PFSH_LAUNCH(name, stream) ::pfsh::LaunchScope pfsh_scope_(name, stream)

// Programmatic dependent launch: a kernel launched with launch_pdl is set up
// while the previous kernel of its stream drains and runs only independent
// work (tables, constants) before pdl_wait(), which returns once that kernel
// has completed and its writes are visible.  Every kernel that can be
// launched this way calls pdl_wait() (also when it reads nothing the previous
// kernel wrote) so that completion stays ordered along the stream.  No kernel
// triggers its dependents early: dependents that became resident early and
// waited held SM resources that the concurrently running fine sweeps need
// (measured: 169 vs 182 iterations/s).  Without a programmatic predecessor
// pdl_wait() is a no-op.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// sticky device status word shared by every object of the library
int *device_status();
// opt-in non-finite check of n doubles (checks.cu): records ST_NUMERIC
int check_finite(const double *x, size_t n, cudaStream_t s);
enum { ST_OK = 0, ST_TIMEOUT = 1, ST_NUMERIC = 2 };

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename R> struct cpx;
template <> struct cpx<double> { typedef double2 t; };
template <> struct cpx<float> { typedef float2 t; };

template <typename C> __host__ __device__ __forceinline__ C mk(double x, double y) {
  C c; c.x = x; c.y = y; return c;
}
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C> __device__ __forceinline__ C times_i(C a) { C r; r.x = -a.y; r.y = a.x; return r; }

// ---------------------------------------------------------------------------
// double <-> float conversions on the integer pipe.  The hardware conversion
// instructions issue on the FP64 pipe, which is narrow on this GPU; these do
// the IEEE-754 format change with integer operations instead.
// d2f: round to nearest even; |x| below the smallest normal float (2^-126)
// becomes a signed zero, overflow gives +-inf, NaN stays NaN.
// f2d: exact (subnormal floats take the hardware path).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float d2f_alu(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // top 23 mantissa bits
  const unsigned rem = lo & 0x1FFFFFFFu;                     // 29 discarded bits
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | ((m | rem) ? 0x400000u : 0u));
  const int fe = e - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
  unsigned r = ((unsigned)fe << 23) | m;
  if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) r += 1u;   // carry may reach +inf: correct
  return __uint_as_float(sign | r);
}

__device__ __forceinline__ double f2d_alu(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  if (e == 0) return m ? (double)f : __hiloint2double((int)sign, 0);
  if (e == 0xffu) return __hiloint2double((int)(sign | 0x7ff00000u | (m >> 3)), (int)(m << 29));
  return __hiloint2double((int)(sign | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

template <typename M> __device__ __forceinline__ double to_double(M x) { return (double)x; }
template <> __device__ __forceinline__ double to_double<float>(float x) { return f2d_alu(x); }
template <typename M> __device__ __forceinline__ M from_double(double x) { return (M)x; }
template <> __device__ __forceinline__ float from_double<float>(double x) { return d2f_alu(x); }

// ---------------------------------------------------------------------------
// triangle indexing
// ---------------------------------------------------------------------------
// packed offset of order m in a degree-T triangle (the ABI layout)
__host__ __device__ __forceinline__ int poff(int T, int m) { return m * (2 * T + 3 - m) / 2; }
// offset of order m in the extended triangle: m <= T, m <= n <= T+1
__host__ __device__ __forceinline__ int eoff(int T, int m) { return m * (T + 2) - m * (m - 1) / 2; }
__host__ __device__ __forceinline__ int ncoef_of(int T) { return (T + 1) * (T + 2) / 2; }
__host__ __device__ __forceinline__ int next_of(int T) { return (T + 1) * (T + 4) / 2; }

// ---------------------------------------------------------------------------
// FFT plan (complex length-N transforms, mixed radix Stockham)
// ---------------------------------------------------------------------------
constexpr int kMaxPasses = 24;
struct FftPlan {
  int N = 0;
  int npass = 0;
  int full = 0;             // offset of the full-circle part of the table
  int radix[kMaxPasses];
  double2 *tw64 = nullptr;  // per-pass twiddles, then exp(-2 pi i e / N), e < N
  float2 *tw32 = nullptr;
};

// ---------------------------------------------------------------------------
// tensor-core Legendre tables (see legendre_tc.cu)
// ---------------------------------------------------------------------------
struct TcChunk {          // one K chunk of one (m, row tile, parity)
  long long off;          // byte offset of its bf16 hi image (lo follows)
  int m, p, kstart, klen; // order, parity of n-m, first K index, K extent (x16)
  int N, row0, nrows;     // MMA N (x16), first row of the tile, valid rows
  int pad;
};
struct TcWork {           // one CTA row tile of order m
  int first, nchunks, N, row0, nrows;
};
// Coriolis term of the implicit part (banded.cuh): coupling table of the
// context and 2 Omega, or {nullptr, 0} when the Coriolis term is explicit
struct CorArgs {
  const double4_32a *ab;   // [ncoef] {alpha_n, beta_n, m/(n(n+1)), 0}
  double tw;               // 2 Omega
};

struct TcDir {
  uint8_t *img = nullptr;
  TcChunk *chunks = nullptr;
  TcWork *work = nullptr;
  int nchunks = 0, ntiles = 0, Nmax = 0;
  size_t img_bytes = 0;
};

// Row tilings of a tensor-core plan: configuration c splits the output rows
// of an order (latitudes for synthesis, degree positions for analysis) into
// ntiles = tile_mult[c] x ceil(rows / 256) tiles; the autotuner of
// legendre_tc.cu picks a configuration per launch width (column blocks of
// 128 real columns, 1..kTcMaxNb).  The tiling splits output rows only, so
// every configuration computes bitwise the same result.
constexpr int kTcConfigs = 2, kTcMaxNb = 8;

// ---------------------------------------------------------------------------
// objects behind the opaque ABI handles
// ---------------------------------------------------------------------------
}  // namespace pfsh

struct sht_plan {
  int T, nlat, nlon, nh, ncoef, ne, max_batch, prec;
  int device;
  std::vector<double> mu, w;        // host copies (ABI sht_info)
  double *d_mu = nullptr;           // [nlat]
  double *d_w = nullptr;            // [nlat]
  double *d_P = nullptr;            // [ne][nh] FP64 P_n^m(mu_j), j north
  float *d_P32 = nullptr;           // [ne][nh] float copy (mixed precisions)
  double *d_eps = nullptr;          // [ne] eps_n^m = sqrt((n^2-m^2)/(4n^2-1)), extended triangle
  double *d_ilap = nullptr;         // [T+2] 1/(n(n+1)) (0 at n = 0)
  float *d_eps32 = nullptr, *d_ilap32 = nullptr;   // float copies for mixed plans
  double *d_rowf = nullptr;         // [nh][2]: 1/(1-mu_j^2), w_j (northern rows)
  float *d_rowf32 = nullptr;        // float copy
  pfsh::FftPlan fft;
  pfsh::TcDir tc[2][pfsh::kTcConfigs];   // [direction: 0 synthesis, 1 analysis][configuration]
  int tc_mult[2][pfsh::kTcConfigs] = {};  // row-tile multiplier of each configuration (0: not built)
  unsigned char tc_pick[2][pfsh::kTcMaxNb] = {};   // configuration per launch width
  // workspace for one pass of at most max_batch fields
  void *ws = nullptr;
  size_t ws_bytes = 0;
  size_t device_bytes = 0;
  // ws carve-up (complex of the plan's real type: double for PFSH_FP64,
  // float otherwise): X [ne][cols], F [T+1][nlat][cols], H [T+1][2][nh][cols],
  // Y [ne][cols]
  void *X = nullptr, *F = nullptr, *H = nullptr, *Y = nullptr;
};

struct swe_ctx {
  sht_plan *plan;
  swe_params prm;
  int max_states;     // states per RHS pass (plan->max_batch / 5)
  // Coriolis term implicit: coupling table [ncoef] and the factor table of
  // swe_implicit_solve [3 ncoef] (banded.cuh band_table_entries)
  double4_32a *d_cor = nullptr;
  double4_32a *d_band_scr = nullptr;
  ~swe_ctx();
};

struct sdc_level {
  swe_ctx *ctx;
  int nodes;          // M + 1
  double dt;
  int max_batch;
  double tau_nodes[16];
  double Q[16][16], QE[16][16], QI[16][16];
  double *d_old = nullptr;   // [M][max_batch][3][ncoef] c128: node-update constants
  double *d_fac = nullptr;   // [M+1][T+1][4] implicit-solve factors per node and degree (solver.cu)
  double4_32a *d_band = nullptr;   // Coriolis implicit: banded-solve factor tables per node [M+1][3 ncoef]
};

// CUDA graphs of iteration blocks keyed by (iterations, last): the first call
// of a key runs eagerly, the second records and launches the graph, later
// calls replay it (see pfasst.cu run_cached).
struct GraphEntry {
  int count = 0, last = 0, calls = 0;
  cudaGraphExec_t exec = nullptr;
  unsigned long long launches = 0;
};
struct GraphCache {
  static constexpr int kMax = 8;
  GraphEntry e[kMax];
};

struct pfasst {
  pfasst_config cfg;
  sht_plan *plan_f = nullptr, *plan_c = nullptr;
  swe_ctx *ctx_f = nullptr, *ctx_c = nullptr;
  sdc_level *lev_f = nullptr, *lev_c = nullptr;
  int Mf, Mc;
  size_t sf, sc;              // doubles per state (3*ncoef*2) fine / coarse
  double *th_f, *fe_f, *fi_f; // [Mf+1][n_ts][state]
  double *th_c, *fe_c, *fi_c; // [Mc+1][n_ts][state]
  double *th_cs, *fe_cs, *fi_cs; // saved restriction (tilde) [Mc+1][n_ts][state]
  double *tau;                // [Mc+1][n_ts][coarse state]
  double *sent;               // [n_ts][fine state]
  double *base_c;             // [n_ts][coarse state] restricted initial value
  double *theta0;             // [fine state]
  double *prev_end = nullptr; // [n_ts][fine state] end values at the last residual check
  double Rt[16][16], Pt[16][16];   // time restriction / interpolation
  // CUDA graphs of iteration blocks, keyed by (iterations, last)
  GraphCache graphs_;
  cudaStream_t cap_stream = nullptr;
  bool graphs = true;
  // Step C runs on its own stream with its own coarse plan/context/level so
  // that it overlaps Steps A and B of later slice groups (see pfasst.cu).
  static constexpr int kMaxGroups = 32;
  int groups = 1;
  cudaStream_t chain_stream = nullptr;
  sht_plan *plan_cc = nullptr;
  swe_ctx *ctx_cc = nullptr;
  sdc_level *lev_cc = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_B[kMaxGroups] = {}, ev_C[kMaxGroups] = {}, ev_R[kMaxGroups] = {};
};

// Independent PFASST instances advanced together (pfasst.cu): each member on
// its own stream (plus its own chain stream), one graph per block.
struct pfasst_ensemble {
  int n = 0;
  pfasst **members = nullptr;
  cudaStream_t *streams = nullptr;
  cudaEvent_t *ev_join = nullptr;
  cudaEvent_t ev_fork = nullptr;
  cudaStream_t cap_stream = nullptr;
  GraphCache graphs_;
  bool graphs = true;
};

namespace pfsh {

// ---------------------------------------------------------------------------
// SDC node-update coefficients (dt folded in); see spectral.cu
// ---------------------------------------------------------------------------
struct SdcCoef {
  double cE[16][16];  // dt (Q - QE') for the "old" right-hand sides
  double cI[16][16];  // dt (Q - QI')
  double nE[16][16];  // dt QE  (new explicit terms, j < i)
  double nI[16][16];  // dt QI  (new implicit terms, j < i)
  double h[16];       // dt QI[i][i]
};
SdcCoef sdc_coef(const sdc_level *l);

inline bool coriolis_implicit(const swe_params &p) { return p.coriolis == PFSH_CORIOLIS_IMPLICIT; }
// the rotation rate seen by the explicit part (eta = zeta + f, or zeta)
inline double omega_explicit(const swe_params &p) { return coriolis_implicit(p) ? 0.0 : p.omega; }
inline CorArgs cor_args(const swe_ctx *c) {
  return coriolis_implicit(c->prm) ? CorArgs{c->d_cor, 2.0 * c->prm.omega} : CorArgs{nullptr, 0.0};
}

// ---------------------------------------------------------------------------
// kernels / launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
int fft_plan_init(FftPlan &f, int N);
void fft_plan_free(FftPlan &f);

// Legendre table generation (FP64 recurrence on the device)
int legendre_table_build(sht_plan *p, cudaStream_t s);
int convert_table_f32(const double *a, float *b, size_t n, cudaStream_t s);

// transforms on the plan's workspace (cols = number of complex columns)
int synth_simt(const sht_plan *p, int cols, cudaStream_t s);      // X -> F
int analysis_simt(const sht_plan *p, int cols, cudaStream_t s);   // H -> Y
int synth_tc(const sht_plan *p, int cols, cudaStream_t s);
int analysis_tc(const sht_plan *p, int cols, cudaStream_t s);
int tc_tables_build(sht_plan *p);   // builds the tilings and runs the autotuner
void tc_tables_free(sht_plan *p);
int tc_tiles_used(const sht_plan *p, int dir, int nb);   // row tiles per order at launch width nb
int synth_small(const sht_plan *p, int cols, cudaStream_t s);
int analysis_small(const sht_plan *p, int cols, cudaStream_t s);
bool small_synth(int cols);
bool small_rhs(int B);
int rhs_small(const sht_plan *p, const double *state, double *fE, double *fI, int B, const swe_params &prm,
              CorArgs cor, cudaStream_t s);
bool small_analysis(int cols);
// launch bookkeeping: kernels replayed by a CUDA graph
void count_launches(unsigned long long n);
unsigned long long launches_so_far();
void g_launches_uncount(unsigned long long n);
bool profiler_on();
// set the dynamic shared-memory limit of a kernel once per process
int ensure_smem(const void *fn, size_t bytes);
// dispatch on the plan's precision
int legendre_synth(const sht_plan *p, int cols, cudaStream_t s);
int legendre_analysis(const sht_plan *p, int cols, cudaStream_t s);
bool uses_tensor_cores(int prec);
int ifft_rows(const sht_plan *p, int cols, void *grid, cudaStream_t s);        // F -> grid
int fft_rows(const sht_plan *p, int cols, const void *grid, cudaStream_t s);   // grid -> H
int grid_rhs(const sht_plan *p, int B, const swe_params &prm, cudaStream_t s,
             bool pdl = false);   // F -> H (RHS)
int ifft_rows_f64_raw(int N, int npass, const int *radix, int full, int T, int nlat, int cols, const double2 *F,
                      const double2 *tw, double *grid, cudaStream_t s);

// spectral pre/post processing
int spec_to_X(const sht_plan *p, const double *spec, int batch, cudaStream_t s);
int Y_to_spec(const sht_plan *p, double *spec, int batch, cudaStream_t s);
// The batch of B states is cnt consecutive states (stride 3 ncoef complex)
// in each of B / cnt groups nstride doubles apart (cnt = 0: one group of B).
int rhs_prep(const sht_plan *p, const double *state, int B, const swe_params &prm, cudaStream_t s, int cnt = 0,
             size_t nstride = 0);
int rhs_assemble(const sht_plan *p, const double *state, double *fE, double *fI, int B,
                 const swe_params &prm, CorArgs cor, cudaStream_t s, int cnt = 0, size_t nstride = 0);

// banded implicit solve of the split with the Coriolis term implicit (banded.cu)
int band_ctx_init(swe_ctx *c);
int band_factor_launch(const swe_ctx *c, double h, double nu, double4_32a *tab, cudaStream_t s);
int band_solve_launch(const swe_ctx *c, const double *b, double *x, double h, int B, cudaStream_t s);
int band_sdc_node_launch(const sdc_level *l, int i, size_t node_stride, const SdcCoef &coef, const double *O,
                         const double *fE, const double *fI, double *theta, int B, cudaStream_t s);
int implicit_solve_launch(int T, const double *b, double *x, double h, int B,
                          const swe_params &prm, cudaStream_t s);

// internal RHS on a contiguous batch (chunks over ctx->max_states)
int rhs_eval(swe_ctx *c, const double *state, double *fE, double *fI, int B, cudaStream_t s);
// F_E, F_I of `nodes` groups of cnt consecutive states, node_stride doubles
// apart (one pass over all nodes x cnt states when the context holds them)
int rhs_eval_nodes(swe_ctx *c, const double *state, double *fE, double *fI, int nodes, int cnt, size_t node_stride,
                   cudaStream_t s);

// SDC pieces: node arrays are [nodes][..] with a node stride (in doubles)
int sdc_sweep_strided(sdc_level *l, double *theta, double *fE, double *fI, const double *tau,
                      size_t node_stride, int B, cudaStream_t s);
int sdc_build_matrices(sdc_level *l, int nodes);
void lagrange_matrix(const double *src, int ns, const double *dst, int nd, double out[16][16]);

// Step C of Algorithm 1 for slices n0..n1-1 with fused per-order launches
// (small.cu); strides in doubles
int chain_sweeps(sdc_level *l, double *th, double *fe, double *fi, const double *tau, size_t node_stride,
                 size_t slice_stride, int n0, int n1, bool recv_first, cudaStream_t s,
                 cudaEvent_t after_first = nullptr);

// PFASST transfer kernels
int restrict_launch(const double *Rt, int nf, int nc, const double *xf, size_t fstride,
                    double *xc, size_t cstride, int Tf, int Tc, int B, cudaStream_t s);

}  // namespace pfsh
