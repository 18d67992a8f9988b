// Allocation-free FP64 synthesis: sht_inverse_noalloc.
//
// Some callers may not allocate device memory at all after start-up (a
// real-time loop under a no-allocation policy, or a host application that
// owns every device byte through its own pool), and so cannot create an
// sht_plan, whose tables and workspace come from cudaMalloc.  This entry point
// serves them: it needs only the caller's input and output buffers.  Its
// working storage -- the Gaussian latitudes, the FFT twiddles and the Fourier
// coefficients F_m(mu_j) -- lives in one file-scope device array of fixed size
// that every GPU which loads this library keeps until the process exits.
// The associated Legendre functions are evaluated on the fly by the same
// FP64 recurrence the plans use to build their tables, so no table is needed.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <string>

#include "fft_core.cuh"
#include "internal.cuh"

namespace pfsh {

constexpr size_t kNoallocScratchBytes = (size_t)4 << 20;   // 4 MiB
constexpr int kNoallocMaxT = 127;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once (host code
// must not pass the symbol itself: on the host it only stands in for the
// device object).  Atomic so that host threads making their first call on
// the same device at the same time do not race (both store the same value).
static std::atomic<void *> g_noalloc_addr[64];

struct PassTable {        // twiddle layout of the FFT passes (fft_core.cuh)
  int npass, full;
  int R[kMaxPasses], Ns[kMaxPasses], off[kMaxPasses];
};

// Gaussian latitudes (northern half, Newton on P_nlat) and FFT twiddles:
// entry off_p + r Ns_p + k of pass p = exp(-2 pi i k r / (Ns_p R_p)), then the
// full circle exp(-2 pi i e / nlon) from offset `full`.
__global__ void k_noalloc_setup(int nlat, int nlon, PassTable pt, double *mu, double2 *tw) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nlat / 2) {
    double x = cospi((t + 0.75) / (nlat + 0.5));
    for (int it = 0; it < 100; ++it) {
      double a = 1.0, b = x;
      for (int k = 1; k < nlat; ++k) {
        const double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
        a = b;
        b = c;
      }
      const double dx = b / (nlat * (x * b - a) / (x * x - 1.0));
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    mu[t] = x;
  }
  if (t < pt.full + nlon) {
    double num, den;
    if (t >= pt.full) {
      num = t - pt.full;
      den = nlon;
    } else {
      int p = 0;
      while (p + 1 < pt.npass && t >= pt.off[p + 1]) ++p;
      const int e = t - pt.off[p], r = e / pt.Ns[p], k = e - r * pt.Ns[p];
      num = (double)k * r;
      den = (double)pt.Ns[p] * pt.R[p];
    }
    double sn, cs;
    sincospi(2.0 * num / den, &sn, &cs);
    tw[t] = make_double2(cs, -sn);
  }
}

// F_m(+-mu_j) = S_0 +- S_1 with S_p = sum_{n-m = p mod 2} c_n^m P_n^m(mu_j),
// P_n^m by the normalised three-term recurrence without rescaling.  For
// T <= 127 on grids with nlat up to a few times T, the sectoral start
// P_m^m(mu_j) stays in the normal double range; on much finer grids it can
// underflow to 0 at the latitudes nearest the poles (e.g. P_127^127 ~ 1e-370
// at the first root when nlat ~ 2000), where the true terms lie below 1e-300
// of the coefficients and do not change the result.
__global__ void k_noalloc_synth(int T, int nlat, int batch, const double *__restrict__ mu,
                                const double2 *__restrict__ spec, double2 *__restrict__ F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (j >= nlat / 2) return;
  const double x = mu[j];
  const double st = sqrt((1.0 - x) * (1.0 + x));
  double pmm = 0.70710678118654752440;   // P_0^0 = 1/sqrt(2)
  for (int k = 1; k <= m; ++k) pmm *= sqrt((2.0 * k + 1.0) / (2.0 * k)) * st;
  const int nc = ncoef_of(T), base = poff(T, m) - m;
  for (int b = 0; b < batch; ++b) {
    const double2 *c = spec + (size_t)b * nc;
    double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
    double p2 = 0.0, p1 = pmm;
    for (int n = m; n <= T; ++n) {
      double p;
      if (n == m) {
        p = pmm;
      } else if (n == m + 1) {
        p = sqrt(2.0 * m + 3.0) * x * p1;
        p2 = p1;
        p1 = p;
      } else {
        const double en = sqrt(((double)n * n - (double)m * m) / (4.0 * n * n - 1.0));
        const double en1 = sqrt(((double)(n - 1) * (n - 1) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0));
        p = (x * p1 - en1 * p2) / en;
        p2 = p1;
        p1 = p;
      }
      double2 v = c[base + n];
      if (m == 0) v.y = 0.0;
      if ((n - m) & 1) {
        s1.x += p * v.x;
        s1.y += p * v.y;
      } else {
        s0.x += p * v.x;
        s0.y += p * v.y;
      }
    }
    F[((size_t)m * nlat + j) * batch + b] = make_double2(s0.x + s1.x, s0.y + s1.y);
    F[((size_t)m * nlat + (nlat - 1 - j)) * batch + b] = make_double2(s0.x - s1.x, s0.y - s1.y);
  }
}

static int radices(int N, int *r, int *np) {
  int n = N, k = 0;
  const int small[] = {4, 2, 3, 5};
  for (int q : small)
    while (n % q == 0) {
      if (k >= kMaxPasses) return -1;
      r[k++] = q;
      n /= q;
    }
  for (int q = 7; n > 1; q += 2)
    while (n % q == 0) {
      if (q > 61 || k >= kMaxPasses) return -1;
      r[k++] = q;
      n /= q;
    }
  *np = k;
  return 0;
}

}  // namespace pfsh

using namespace pfsh;

extern "C" int sht_inverse_noalloc(int T, int nlat, int nlon, const double *spec, double *grid, int batch,
                                   pfsh_stream_t stream) {
  if (T < 1 || T > kNoallocMaxT || nlat % 2 || nlat < T + 2 || nlon % 2 || nlon <= 2 * (T + 1) || batch < 0)
    return fail(PFSH_EINVAL, "sht_inverse_noalloc: need 1 <= T <= 127, nlat even >= T+2, nlon even > 2(T+1)");
  if (batch == 0) return PFSH_OK;
  if (!spec || !grid) return fail(PFSH_EINVAL, "sht_inverse_noalloc: NULL buffer");
  int rad[kMaxPasses], npass = 0;
  if (!ct_radix_list(nlon, rad, &npass) && radices(nlon, rad, &npass))
    return fail(PFSH_EINVAL, "sht_inverse_noalloc: nlon has a prime factor above 61");
  PassTable pt{};
  pt.npass = npass;
  {
    int Ns = 1, off = 0;
    for (int p = 0; p < npass; ++p) {
      pt.R[p] = rad[p];
      pt.Ns[p] = Ns;
      pt.off[p] = off;
      off += rad[p] * Ns;
      Ns *= rad[p];
    }
    pt.full = off;
  }
  const int ntw = pt.full + nlon;
  // the inverse longitude transform holds two padded rows per block in shared memory
  const size_t fft_smem = 2 * (size_t)padded(nlon) * sizeof(double2);
  if (fft_smem > (size_t)227 * 1024)
    return fail(PFSH_EINVAL, "sht_inverse_noalloc: nlon too long for the shared-memory row transform");
  // scratch: mu [nlat/2] | twiddles [nlon] | F [T+1][nlat][batch], each 256-byte aligned
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t o_tw = up((size_t)(nlat / 2) * sizeof(double));
  const size_t o_F = o_tw + up((size_t)ntw * sizeof(double2));
  const size_t need = o_F + (size_t)(T + 1) * nlat * batch * sizeof(double2);
  if (need > kNoallocScratchBytes)
    return fail(PFSH_EINVAL, "sht_inverse_noalloc: (T+1)*nlat*batch*16 bytes plus nodes and twiddles exceed the "
                             "4 MiB scratch; use fewer fields per call");
  int dev = 0;
  PFSH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(PFSH_EUNSUPPORTED, "sht_inverse_noalloc: device index");
  void *addr = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!addr) {
    cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "sht_inverse_noalloc: cudaGetSymbolAddress");
    g_noalloc_addr[dev].store(addr, std::memory_order_release);
  }
  unsigned char *base = (unsigned char *)addr;
  double *mu = (double *)base;
  double2 *tw = (double2 *)(base + o_tw);
  double2 *F = (double2 *)(base + o_F);
  cudaStream_t s = (cudaStream_t)stream;
  {
    const int n = std::max(nlat / 2, ntw);
    PFSH_LAUNCH("k_noalloc_setup", s);
    k_noalloc_setup<<<(n + 127) / 128, 128, 0, s>>>(nlat, nlon, pt, mu, tw);
  }
  PFSH_CHECK_LAUNCH("k_noalloc_setup");
  {
    PFSH_LAUNCH("k_noalloc_synth", s);
    k_noalloc_synth<<<dim3((nlat / 2 + 63) / 64, T + 1), 64, 0, s>>>(T, nlat, batch, mu, (const double2 *)spec, F);
  }
  PFSH_CHECK_LAUNCH("k_noalloc_synth");
  return ifft_rows_f64_raw(nlon, npass, rad, pt.full, T, nlat, batch, F, tw, grid, s);
}
