// Transform plan: Gaussian grid, associated Legendre table, FFT plan,
// workspace; the sht_* entry points; error and status plumbing.
//
// Section 3 of the paper: Gaussian latitudes mu = sin(phi) with Gauss
// weights, normalised associated Legendre functions, two-step transform
// (DFT in longitude, Gauss-Legendre quadrature in latitude).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "fft_core.cuh"
#include "internal.cuh"

namespace pfsh {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return PFSH_ECUDA;
}

// One status word per device, allocated on first use.
static int *g_status[64] = {nullptr};

int *device_status() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!g_status[dev]) {
    int *p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
    g_status[dev] = p;
  }
  return g_status[dev];
}

// ---------------------------------------------------------------------------
// Gaussian latitudes and weights (host, FP64 Newton iteration on P_nlat)
// ---------------------------------------------------------------------------
static void legendre_pair(int N, double x, double *pN, double *pNm1) {
  double a = 1.0, b = x;  // P_0, P_1
  if (N == 0) { *pN = 1.0; *pNm1 = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
    a = b;
    b = c;
  }
  *pN = b;
  *pNm1 = a;
}

static void gauss_grid(int nlat, std::vector<double> &mu, std::vector<double> &w) {
  mu.assign(nlat, 0.0);
  w.assign(nlat, 0.0);
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < nlat / 2; ++j) {
    double x = std::cos(pi * (j + 0.75) / (nlat + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, q;
      legendre_pair(nlat, x, &p, &q);
      double dp = nlat * (x * p - q) / (x * x - 1.0);
      double dx = p / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double p, q;
    legendre_pair(nlat, x, &p, &q);
    double dp = nlat * (x * p - q) / (x * x - 1.0);
    double wt = 2.0 / ((1.0 - x) * (1.0 + x) * dp * dp);
    mu[j] = x;
    mu[nlat - 1 - j] = -x;
    w[j] = wt;
    w[nlat - 1 - j] = wt;
  }
}

// ---------------------------------------------------------------------------
// Associated Legendre table (device FP64 recurrence in n, per (m, j))
// ---------------------------------------------------------------------------
// The sectoral start P_m^m(mu_j) = (1/sqrt 2) prod_{k<=m} sqrt((2k+1)/2k)
// (1-mu_j^2)^{m/2} is carried as mantissa * 2^exponent (computed on the
// host, exact power-of-two rescaling); the n-recurrence
//   P_{m+1}^m = sqrt(2m+3) mu P_m^m,
//   P_n^m = (mu P_{n-1}^m - eps_{n-1}^m P_{n-2}^m) / eps_n^m,
//   eps_n^m = sqrt((n^2-m^2)/(4n^2-1)),
// rescales the mantissa by 2^-400 whenever it exceeds 2^400.  Values whose
// exponent is below the double range become exact zeros.
__global__ void k_legendre_table(int T, int nh, const double *__restrict__ mu,
                                 const double *__restrict__ pmm_mant,
                                 const int *__restrict__ pmm_exp, double *__restrict__ P) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int m = blockIdx.y;
  if (j >= nh) return;
  const double x = mu[j];
  double p1 = pmm_mant[m * nh + j];
  double p2 = 0.0;
  int e = pmm_exp[m * nh + j];
  double *out = P + (size_t)eoff(T, m) * nh + j;
  for (int n = m; n <= T + 1; ++n) {
    if (n == m + 1) {
      double p = sqrt(2.0 * m + 3.0) * x * p1;
      p2 = p1;
      p1 = p;
    } else if (n > m + 1) {
      double en = sqrt(((double)n * n - (double)m * m) / (4.0 * n * n - 1.0));
      double en1 = sqrt(((double)(n - 1) * (n - 1) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0));
      double p = (x * p1 - en1 * p2) / en;
      p2 = p1;
      p1 = p;
    }
    if (fabs(p1) > 0x1p400) {
      p1 = scalbn(p1, -400);
      p2 = scalbn(p2, -400);
      e += 400;
    }
    out[(size_t)(n - m) * nh] = (e < -1200) ? 0.0 : scalbn(p1, e);
  }
}

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ b, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

int convert_table_f32(const double *a, float *b, size_t n, cudaStream_t s) {
  {
    PFSH_LAUNCH("k_to_f32", s);
    k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, n);
  }
  PFSH_CHECK_LAUNCH("k_to_f32");
  PFSH_CUDA(cudaStreamSynchronize(s));
  return PFSH_OK;
}

bool uses_tensor_cores(int prec) {
  return prec == PFSH_BF16 || prec == PFSH_FP16 || prec == PFSH_BF16X3 || prec == PFSH_BF16X6;
}

// Batches of one or two states (the serial coarse chain of PFASST) take
// latency-oriented CUDA-core kernels (fp64 for FP64 plans, fp32 otherwise):
// a 128-row tensor-core tile would be at least 94% padding there.
int legendre_synth(const sht_plan *p, int cols, cudaStream_t s) {
  if (small_synth(cols)) return synth_small(p, cols, s);
  return uses_tensor_cores(p->prec) ? synth_tc(p, cols, s) : synth_simt(p, cols, s);
}

int legendre_analysis(const sht_plan *p, int cols, cudaStream_t s) {
  if (small_analysis(cols)) return analysis_small(p, cols, s);
  return uses_tensor_cores(p->prec) ? analysis_tc(p, cols, s) : analysis_simt(p, cols, s);
}

int legendre_table_build(sht_plan *p, cudaStream_t s) {
  const int T = p->T, nh = p->nh;
  std::vector<double> mant((size_t)(T + 1) * nh);
  std::vector<int> ex((size_t)(T + 1) * nh);
  for (int j = 0; j < nh; ++j) {
    const double x = p->mu[j];
    const double st = std::sqrt((1.0 - x) * (1.0 + x));
    int e0;
    double v = std::frexp(1.0 / std::sqrt(2.0), &e0);
    int e = e0;
    for (int m = 0; m <= T; ++m) {
      if (m > 0) {
        int de;
        v = std::frexp(v * std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * st, &de);
        e += de;
      }
      mant[(size_t)m * nh + j] = v;
      ex[(size_t)m * nh + j] = e;
    }
  }
  double *d_mant = nullptr;
  int *d_ex = nullptr;
  PFSH_CUDA(cudaMalloc(&d_mant, mant.size() * sizeof(double)));
  PFSH_CUDA(cudaMalloc(&d_ex, ex.size() * sizeof(int)));
  PFSH_CUDA(cudaMemcpy(d_mant, mant.data(), mant.size() * sizeof(double), cudaMemcpyHostToDevice));
  PFSH_CUDA(cudaMemcpy(d_ex, ex.data(), ex.size() * sizeof(int), cudaMemcpyHostToDevice));
  dim3 grid((nh + 127) / 128, T + 1);
  {
    PFSH_LAUNCH("k_legendre_table", s);
    k_legendre_table<<<grid, 128, 0, s>>>(T, nh, p->d_mu, d_mant, d_ex, p->d_P);
  }
  PFSH_CHECK_LAUNCH("k_legendre_table");
  PFSH_CUDA(cudaStreamSynchronize(s));
  cudaFree(d_mant);
  cudaFree(d_ex);
  return PFSH_OK;
}

// ---------------------------------------------------------------------------
// FFT plan
// ---------------------------------------------------------------------------
int fft_plan_init(FftPlan &f, int N) {
  f.N = N;
  f.npass = 0;
  if (!ct_radix_list(N, f.radix, &f.npass)) {
    int n = N;
    const int small[] = {4, 2, 3, 5};
    for (int r : small) {
      while (n % r == 0) {
        if (f.npass >= kMaxPasses) return fail(PFSH_EINVAL, "FFT length has too many factors");
        f.radix[f.npass++] = r;
        n /= r;
      }
    }
    for (int r = 7; n > 1; r += 2) {
      while (n % r == 0) {
        if (r > 61) return fail(PFSH_EINVAL, "FFT length has a prime factor above 61");
        if (f.npass >= kMaxPasses) return fail(PFSH_EINVAL, "FFT length has too many factors");
        f.radix[f.npass++] = r;
        n /= r;
      }
    }
  }
  // per-pass twiddles (entry r*Ns + k of pass (R, Ns) = exp(-2 pi i k r/(Ns R)))
  // followed by the full circle exp(-2 pi i e/N), e < N; host libm in double
  std::vector<double2> t64;
  const double two_pi = 6.28318530717958647692;
  int Ns = 1;
  for (int p = 0; p < f.npass; ++p) {
    const int R = f.radix[p];
    for (int r = 0; r < R; ++r)
      for (int k = 0; k < Ns; ++k) {
        const double ang = two_pi * (double)(k * r) / (double)(Ns * R);
        t64.push_back(make_double2(std::cos(ang), -std::sin(ang)));
      }
    Ns *= R;
  }
  f.full = (int)t64.size();
  for (int e = 0; e < N; ++e) {
    const double ang = two_pi * (double)e / (double)N;
    t64.push_back(make_double2(std::cos(ang), -std::sin(ang)));
  }
  std::vector<float2> t32(t64.size());
  for (size_t i = 0; i < t64.size(); ++i) t32[i] = make_float2((float)t64[i].x, (float)t64[i].y);
  PFSH_CUDA(cudaMalloc(&f.tw64, t64.size() * sizeof(double2)));
  PFSH_CUDA(cudaMalloc(&f.tw32, t32.size() * sizeof(float2)));
  PFSH_CUDA(cudaMemcpy(f.tw64, t64.data(), t64.size() * sizeof(double2), cudaMemcpyHostToDevice));
  PFSH_CUDA(cudaMemcpy(f.tw32, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice));
  return PFSH_OK;
}

void fft_plan_free(FftPlan &f) {
  if (f.tw64) cudaFree(f.tw64);
  if (f.tw32) cudaFree(f.tw32);
  f.tw64 = nullptr;
  f.tw32 = nullptr;
}

}  // namespace pfsh

using namespace pfsh;

// ---------------------------------------------------------------------------
// ABI: plans
// ---------------------------------------------------------------------------
static void plan_free(sht_plan *p) {
  if (!p) return;
  if (p->d_mu) cudaFree(p->d_mu);
  if (p->d_w) cudaFree(p->d_w);
  if (p->d_P) cudaFree(p->d_P);
  if (p->d_P32) cudaFree(p->d_P32);
  if (p->d_eps) cudaFree(p->d_eps);
  if (p->d_ilap) cudaFree(p->d_ilap);
  if (p->d_eps32) cudaFree(p->d_eps32);
  if (p->d_rowf) cudaFree(p->d_rowf);
  if (p->d_rowf32) cudaFree(p->d_rowf32);
  if (p->d_ilap32) cudaFree(p->d_ilap32);
  if (p->ws) cudaFree(p->ws);
  fft_plan_free(p->fft);
  tc_tables_free(p);
  delete p;
}

extern "C" int sht_plan_create(sht_plan **out, int T, int nlat, int nlon, int max_batch, int prec) {
  if (!out) return fail(PFSH_EINVAL, "sht_plan_create: out is NULL");
  *out = nullptr;
  if (T < 1) return fail(PFSH_EINVAL, "sht_plan_create: T must be >= 1");
  if (nlat % 2 != 0 || nlat < T + 2) return fail(PFSH_EINVAL, "sht_plan_create: nlat must be even and >= T+2");
  if (nlon % 2 != 0 || nlon <= 2 * (T + 1)) return fail(PFSH_EINVAL, "sht_plan_create: nlon must be even and > 2(T+1)");
  if (max_batch < 1) return fail(PFSH_EINVAL, "sht_plan_create: max_batch must be >= 1");
  if (prec != PFSH_FP64 && prec != PFSH_FP32 && !uses_tensor_cores(prec))
    return fail(PFSH_EUNSUPPORTED, "sht_plan_create: precision not compiled into the library");
  sht_plan *p = new (std::nothrow) sht_plan();
  if (!p) return fail(PFSH_ENOMEM, "sht_plan_create: host allocation");
  p->T = T;
  p->nlat = nlat;
  p->nlon = nlon;
  p->nh = nlat / 2;
  p->ncoef = ncoef_of(T);
  p->ne = next_of(T);
  p->max_batch = max_batch;
  p->prec = prec;
  cudaGetDevice(&p->device);
  gauss_grid(nlat, p->mu, p->w);
  int rc = fft_plan_init(p->fft, nlon);
  if (rc != PFSH_OK) { plan_free(p); return rc; }
  auto alloc = [&](void **ptr, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PFSH_ENOMEM, "sht_plan_create: cudaMalloc of " + std::to_string(bytes) + " bytes");
    }
    p->device_bytes += bytes;
    return PFSH_OK;
  };
  if ((rc = alloc((void **)&p->d_mu, nlat * sizeof(double))) ||
      (rc = alloc((void **)&p->d_w, nlat * sizeof(double))) ||
      (rc = alloc((void **)&p->d_P, (size_t)p->ne * p->nh * sizeof(double)))) {
    plan_free(p);
    return rc;
  }
  if ((rc = alloc((void **)&p->d_eps, (size_t)p->ne * sizeof(double))) ||
      (rc = alloc((void **)&p->d_ilap, (size_t)(T + 2) * sizeof(double)))) {
    plan_free(p);
    return rc;
  }
  {
    std::vector<double> eps(p->ne), ilap(T + 2, 0.0);
    for (int m = 0; m <= T; ++m)
      for (int n = m; n <= T + 1; ++n)
        eps[eoff(T, m) + (n - m)] =
            n > m ? std::sqrt(((double)n * n - (double)m * m) / (4.0 * (double)n * n - 1.0)) : 0.0;
    for (int n = 1; n <= T + 1; ++n) ilap[n] = 1.0 / ((double)n * (n + 1));
    cudaMemcpy(p->d_eps, eps.data(), eps.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_ilap, ilap.data(), ilap.size() * sizeof(double), cudaMemcpyHostToDevice);
    std::vector<float> eps32(eps.begin(), eps.end()), ilap32(ilap.begin(), ilap.end());
    if ((rc = alloc((void **)&p->d_eps32, eps32.size() * sizeof(float))) ||
        (rc = alloc((void **)&p->d_ilap32, ilap32.size() * sizeof(float)))) {
      plan_free(p);
      return rc;
    }
    cudaMemcpy(p->d_eps32, eps32.data(), eps32.size() * sizeof(float), cudaMemcpyHostToDevice);
    std::vector<double> rowf((size_t)p->nh * 2);
    for (int j = 0; j < p->nh; ++j) {
      const double x = p->mu[j];
      rowf[2 * j] = 1.0 / ((1.0 - x) * (1.0 + x));
      rowf[2 * j + 1] = p->w[j];
    }
    std::vector<float> rowf32(rowf.begin(), rowf.end());
    if ((rc = alloc((void **)&p->d_rowf, rowf.size() * sizeof(double))) ||
        (rc = alloc((void **)&p->d_rowf32, rowf32.size() * sizeof(float)))) {
      plan_free(p);
      return rc;
    }
    cudaMemcpy(p->d_rowf, rowf.data(), rowf.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_rowf32, rowf32.data(), rowf32.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_ilap32, ilap32.data(), ilap32.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  cudaMemcpy(p->d_mu, p->mu.data(), nlat * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_w, p->w.data(), nlat * sizeof(double), cudaMemcpyHostToDevice);
  // workspace: X [ne][cols], F [T+1][nlat][cols], H [T+1][2][nh][cols], Y [ne][cols]
  const size_t cols = (size_t)max_batch;
  const size_t celem = prec == PFSH_FP64 ? 16 : 8;
  // each region starts on a 256-byte boundary (bulk copies read 16-byte aligned rows)
  auto up256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t bX = up256((size_t)p->ne * cols * celem);
  const size_t bF = up256((size_t)(T + 1) * nlat * cols * celem);
  const size_t bH = bF;
  const size_t bY = bX;
  p->ws_bytes = bX + bF + bH + bY;
  if ((rc = alloc(&p->ws, p->ws_bytes))) { plan_free(p); return rc; }
  char *base = (char *)p->ws;
  p->X = base;
  p->F = base + bX;
  p->H = base + bX + bF;
  p->Y = base + bX + bF + bH;
  if ((rc = legendre_table_build(p, 0)) != PFSH_OK) { plan_free(p); return rc; }
  if (uses_tensor_cores(prec)) {
    if ((rc = tc_tables_build(p)) != PFSH_OK) { plan_free(p); return rc; }
  }
  if (prec != PFSH_FP64) {
    const size_t n = (size_t)p->ne * p->nh;
    if ((rc = alloc((void **)&p->d_P32, n * sizeof(float)))) { plan_free(p); return rc; }
    if ((rc = convert_table_f32(p->d_P, p->d_P32, n, 0))) { plan_free(p); return rc; }
  }
  if (!device_status()) { plan_free(p); return fail(PFSH_ENOMEM, "status word"); }
  *out = p;
  return PFSH_OK;
}

extern "C" int sht_plan_destroy(sht_plan *p) {
  if (!p) return PFSH_OK;
  cudaDeviceSynchronize();
  plan_free(p);
  return PFSH_OK;
}

extern "C" int sht_plan_query(const sht_plan *p, sht_info *info) {
  if (!p || !info) return fail(PFSH_EINVAL, "sht_plan_query: NULL argument");
  info->T = p->T;
  info->nlat = p->nlat;
  info->nlon = p->nlon;
  info->ncoef = p->ncoef;
  info->max_batch = p->max_batch;
  info->prec = p->prec;
  info->device_bytes = p->device_bytes;
  info->mu = p->mu.data();
  info->w = p->w.data();
  for (int dir = 0; dir < 2; ++dir)
    for (int nb = 1; nb <= 8; ++nb) info->tc_tiles[dir][nb - 1] = tc_tiles_used(p, dir, nb);
  return PFSH_OK;
}

extern "C" int sht_inverse(sht_plan *p, const double *spec, void *grid, int batch, pfsh_stream_t stream) {
  if (!p || batch < 0 || (batch > 0 && (!spec || !grid))) return fail(PFSH_EINVAL, "sht_inverse: invalid argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t gelem = p->prec == PFSH_FP64 ? 8 : 4;
  for (int b0 = 0; b0 < batch; b0 += p->max_batch) {
    int nb = std::min(p->max_batch, batch - b0);
    int rc;
    if ((rc = spec_to_X(p, spec + (size_t)b0 * p->ncoef * 2, nb, s))) return rc;
    if ((rc = legendre_synth(p, nb, s))) return rc;
    if ((rc = ifft_rows(p, nb, (char *)grid + (size_t)b0 * p->nlat * p->nlon * gelem, s))) return rc;
  }
  return PFSH_OK;
}

extern "C" int sht_forward(sht_plan *p, const void *grid, double *spec, int batch, pfsh_stream_t stream) {
  if (!p || batch < 0 || (batch > 0 && (!spec || !grid))) return fail(PFSH_EINVAL, "sht_forward: invalid argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t gelem = p->prec == PFSH_FP64 ? 8 : 4;
  for (int b0 = 0; b0 < batch; b0 += p->max_batch) {
    int nb = std::min(p->max_batch, batch - b0);
    int rc;
    if ((rc = fft_rows(p, nb, (const char *)grid + (size_t)b0 * p->nlat * p->nlon * gelem, s))) return rc;
    if ((rc = legendre_analysis(p, nb, s))) return rc;
    if ((rc = Y_to_spec(p, spec + (size_t)b0 * p->ncoef * 2, nb, s))) return rc;
  }
  return PFSH_OK;
}

extern "C" int pfsh_sync_status(pfsh_stream_t stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pfsh_sync_status");
  int *d = device_status();
  if (!d) return PFSH_OK;
  int h = 0;
  e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "pfsh_sync_status");
  if (h != ST_OK) {
    cudaMemset(d, 0, sizeof(int));
    if (h == ST_TIMEOUT) return fail(PFSH_ETIMEOUT, "a bounded device-side wait gave up");
    return fail(PFSH_ENUMERIC, "device-side check found a non-finite value");
  }
  return PFSH_OK;
}

extern "C" const char *pfsh_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// launch counting and the opt-in event profiler
// ---------------------------------------------------------------------------
#include <atomic>
#include <map>
#include <mutex>

namespace pfsh {
namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
struct ProfRec {
  const char *name;
  cudaEvent_t a, b;
};
std::vector<ProfRec> g_prof;
}  // namespace

void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(); }
// launches recorded during a stream capture did not run; the replays count them
void g_launches_uncount(unsigned long long n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
bool profiler_on() { return g_prof_on.load() != 0; }

static std::mutex g_smem_mu;
static std::map<const void *, size_t> g_smem_set;

int ensure_smem(const void *fn, size_t bytes) {
  if (bytes <= 48 * 1024) return PFSH_OK;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  const void *key = (const char *)fn + dev;   // per device
  auto it = g_smem_set.find(key);
  if (it != g_smem_set.end() && it->second >= bytes) return PFSH_OK;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
  g_smem_set[key] = bytes;
  return PFSH_OK;
}

LaunchScope::LaunchScope(const char *n, cudaStream_t s) : name(n), stream(s), slot(-1) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  ProfRec r{n, nullptr, nullptr};
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
  cudaEventRecord(r.a, s);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  slot = (int)g_prof.size();
  g_prof.push_back(r);
}

LaunchScope::~LaunchScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < (int)g_prof.size()) cudaEventRecord(g_prof[slot].b, stream);
}

static void prof_clear() {
  for (auto &r : g_prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.clear();
}

}  // namespace pfsh

extern "C" unsigned long long pfsh_kernel_launches(void) { return pfsh::g_launches.load(); }

extern "C" int pfsh_profiler_enable(int on) {
  std::lock_guard<std::mutex> lk(pfsh::g_prof_mu);
  if (on) pfsh::prof_clear();
  pfsh::g_prof_on.store(on ? 1 : 0);
  return PFSH_OK;
}

extern "C" int pfsh_profiler_report(char *buf, size_t n) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(pfsh::g_prof_mu);
  std::map<std::string, std::pair<long, double>> acc;
  for (auto &r : pfsh::g_prof) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
    auto &e = acc[r.name];
    e.first += 1;
    e.second += ms;
  }
  std::string out = "{";
  for (auto &kv : acc) {
    if (out.size() > 1) out += ", ";
    char tmp[256];
    snprintf(tmp, sizeof(tmp), "\"%s\": [%ld, %.6f]", kv.first.c_str(), kv.second.first, kv.second.second);
    out += tmp;
  }
  out += "}";
  if (buf && n) {
    size_t k = std::min(n - 1, out.size());
    memcpy(buf, out.data(), k);
    buf[k] = 0;
  }
  return (int)out.size() + 1;
}
