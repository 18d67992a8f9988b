// Longitude transforms and grid products (Section 3 two-step transform;
// Section 2 nonlinear operator evaluated on the grid).
//
// A northern row j and its mirror nlat-1-j are transformed together: the
// complex sequence z_k = north_k + i south_k has spectrum Z_m = N_m + i S_m
// and Z_{N-m} = conj(N_m) + i conj(S_m), so one complex FFT of length nlon
// serves two real rows.  The FFT is a mixed-radix Stockham transform in
// shared memory (radices 4, 2, 3, 5 unrolled; other primes up to 61 by a
// direct DFT), with twiddles exp(-2 pi i e/N) generated on the host in FP64.
#include <algorithm>

#include "fft_core.cuh"
#include "internal.cuh"

namespace pfsh {

static FftArgs fft_args(const FftPlan &f) {
  FftArgs a;
  a.N = f.N;
  a.npass = f.npass;
  a.full = f.full;
  for (int i = 0; i < kMaxPasses; ++i) a.radix[i] = i < f.npass ? f.radix[i] : 1;
  return a;
}

// ---------------------------------------------------------------------------
// inverse: F[m][lat][col] -> grid[col][lat][lon]
// ---------------------------------------------------------------------------
template <typename Rl, typename Shape>
__global__ void k_ifft_rows(FftArgs f, int T, int nlat, int cols, const typename cpx<Rl>::t *__restrict__ F,
                            const typename cpx<Rl>::t *__restrict__ tw, Rl *__restrict__ grid) {
  typedef typename cpx<Rl>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = Shape::n(f), NP = padded(N);
  C *a = reinterpret_cast<C *>(smem_raw);
  C *b = a + NP;
  const int j = blockIdx.y, col = blockIdx.x, js = nlat - 1 - j;
  for (int k = threadIdx.x; k < N; k += blockDim.x) a[sidx(k)] = mk<C>(0.0, 0.0);
  __syncthreads();
  for (int m = threadIdx.x; m <= T; m += blockDim.x) {
    C fn = F[((size_t)m * nlat + j) * cols + col];
    C fs = F[((size_t)m * nlat + js) * cols + col];
    if (m == 0) {
      a[0] = mk<C>(fn.x, fs.x);
    } else {
      a[sidx(m)] = mk<C>(fn.x - fs.y, fn.y + fs.x);
      a[sidx(N - m)] = mk<C>(fn.x + fs.y, -fn.y + fs.x);
    }
  }
  __syncthreads();
  C *r = Shape::run(f, a, b, 1, tw, true);
  Rl *gn = grid + ((size_t)col * nlat + j) * N;
  Rl *gs = grid + ((size_t)col * nlat + js) * N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    C z = r[sidx(k)];
    gn[k] = z.x;
    gs[k] = z.y;
  }
}

// ---------------------------------------------------------------------------
// forward: grid[col][lat][lon] -> H[m][parity][j][col] (weights and 1/N applied)
// ---------------------------------------------------------------------------
template <typename C, typename Rl>
__device__ __forceinline__ void unpack_write(const C *Z, int N, int T, int j, int nh, int cols, int col,
                                             Rl wj, C *__restrict__ H) {
  const Rl half = (Rl)0.5 / (Rl)N;
  for (int m = threadIdx.x; m <= T; m += blockDim.x) {
    C zm = Z[sidx(m)];
    C zc = cconj(Z[sidx(m == 0 ? 0 : N - m)]);
    C gn = half * (zm + zc);              // north spectrum
    C gs = half * times_i(zc - zm);       // south spectrum: (zm - zc) / (2i)
    C he = wj * (gn + gs), ho = wj * (gn - gs);
    H[(((size_t)m * 2 + 0) * nh + j) * cols + col] = he;
    H[(((size_t)m * 2 + 1) * nh + j) * cols + col] = ho;
  }
}

template <typename Rl, typename Shape>
__global__ void k_fft_rows(FftArgs f, int T, int nlat, int cols, const Rl *__restrict__ grid,
                           const double *__restrict__ w, const typename cpx<Rl>::t *__restrict__ tw,
                           typename cpx<Rl>::t *__restrict__ H) {
  typedef typename cpx<Rl>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = Shape::n(f), NP = padded(N);
  C *a = reinterpret_cast<C *>(smem_raw);
  C *b = a + NP;
  const int j = blockIdx.y, col = blockIdx.x, js = nlat - 1 - j;
  const Rl *gn = grid + ((size_t)col * nlat + j) * N;
  const Rl *gs = grid + ((size_t)col * nlat + js) * N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) a[sidx(k)] = mk<C>(gn[k], gs[k]);
  __syncthreads();
  C *r = Shape::run(f, a, b, 1, tw, false);
  unpack_write<C, Rl>(r, N, T, j, nlat / 2, cols, col, (Rl)w[j], H);
}

// ---------------------------------------------------------------------------
// RHS grid stage: 4 spectra (eta, Phi', U, V) per state -> 5 products
//   A1 = eta U/(1-mu^2), B1 = eta V/(1-mu^2), A2 = Phi' U/(1-mu^2),
//   B2 = Phi' V/(1-mu^2), E = (U^2+V^2)/(2(1-mu^2))
// F columns: b*4 + f ; H columns: b*5 + f
// ---------------------------------------------------------------------------
template <typename Rl, typename Shape>
__global__ void __launch_bounds__(256) k_grid_rhs(FftArgs f, int T, int nlat, int B,
                                                  const typename cpx<Rl>::t *__restrict__ F,
                                                  const Rl *__restrict__ rowf,
                                                  const typename cpx<Rl>::t *__restrict__ tw,
                                                  typename cpx<Rl>::t *__restrict__ H, bool center) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  grid_rhs_body<Rl, Shape>(f, T, nlat, B, blockIdx.y, blockIdx.x, F, rowf, tw, H,
                           reinterpret_cast<typename cpx<Rl>::t *>(smem_raw), center);
}

// One block per latitude pair and state holds 6 padded transforms (up to
// 196 KB at nlon = 3840 in fp32), so a single block runs per SM: 512 threads
// (measured at T1279: 34.8 ms of grid stage per PFASST iteration, 36.8 with
// 256 threads).
constexpr int kLongThreads = 512;

template <typename Rl, typename Shape>
__global__ void __launch_bounds__(kLongThreads) k_grid_rhs_long(FftArgs f, int T, int nlat, int B,
                                                       const typename cpx<Rl>::t *__restrict__ F,
                                                       const Rl *__restrict__ rowf,
                                                       const typename cpx<Rl>::t *__restrict__ tw,
                                                       typename cpx<Rl>::t *__restrict__ H, bool center) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  grid_rhs_body_long<Rl, Shape>(f, T, nlat, B, blockIdx.y, blockIdx.x, F, rowf, tw, H,
                                reinterpret_cast<typename cpx<Rl>::t *>(smem_raw), center);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int set_smem(const void *fn, size_t bytes) { return ensure_smem(fn, bytes); }

template <typename Rl>
static int ifft_launch(const FftArgs &f, int T, int nlat, int cols, const typename cpx<Rl>::t *F,
                       const typename cpx<Rl>::t *tw, Rl *grid, cudaStream_t s) {
  const size_t sm = 2 * (size_t)padded(f.N) * sizeof(typename cpx<Rl>::t);
  return with_shape(f.N, [&]<typename Shape>() -> int {
    int rc = set_smem((const void *)k_ifft_rows<Rl, Shape>, sm);
    if (rc) return rc;
    {
      PFSH_LAUNCH("k_ifft_rows", s);
      k_ifft_rows<Rl, Shape><<<dim3(cols, nlat / 2), 256, sm, s>>>(f, T, nlat, cols, F, tw, grid);
    }
    PFSH_CHECK_LAUNCH("k_ifft_rows");
    return PFSH_OK;
  });
}

int ifft_rows(const sht_plan *p, int cols, void *grid, cudaStream_t s) {
  FftArgs f = fft_args(p->fft);
  if (p->prec == PFSH_FP64)
    return ifft_launch<double>(f, p->T, p->nlat, cols, (const double2 *)p->F, p->fft.tw64, (double *)grid, s);
  return ifft_launch<float>(f, p->T, p->nlat, cols, (const float2 *)p->F, p->fft.tw32, (float *)grid, s);
}

// Inverse longitude transform of F[m][lat][cols] (complex fp64) into
// grid[cols][lat][lon] with caller-supplied radix list and twiddle table (the
// per-pass layout of fft_core.cuh, full circle at offset `full`); used by the
// allocation-free synthesis entry point.
int ifft_rows_f64_raw(int N, int npass, const int *radix, int full, int T, int nlat, int cols, const double2 *F,
                      const double2 *tw, double *grid, cudaStream_t s) {
  FftArgs f;
  f.N = N;
  f.npass = npass;
  f.full = full;
  for (int i = 0; i < kMaxPasses; ++i) f.radix[i] = i < npass ? radix[i] : 1;
  return ifft_launch<double>(f, T, nlat, cols, F, tw, grid, s);
}

template <typename Rl>
static int fft_launch(const FftArgs &f, int T, int nlat, int cols, const Rl *grid, const double *w,
                      const typename cpx<Rl>::t *tw, typename cpx<Rl>::t *H, cudaStream_t s) {
  const size_t sm = 2 * (size_t)padded(f.N) * sizeof(typename cpx<Rl>::t);
  return with_shape(f.N, [&]<typename Shape>() -> int {
    int rc = set_smem((const void *)k_fft_rows<Rl, Shape>, sm);
    if (rc) return rc;
    {
      PFSH_LAUNCH("k_fft_rows", s);
      k_fft_rows<Rl, Shape><<<dim3(cols, nlat / 2), 256, sm, s>>>(f, T, nlat, cols, grid, w, tw, H);
    }
    PFSH_CHECK_LAUNCH("k_fft_rows");
    return PFSH_OK;
  });
}

int fft_rows(const sht_plan *p, int cols, const void *grid, cudaStream_t s) {
  FftArgs f = fft_args(p->fft);
  if (p->prec == PFSH_FP64)
    return fft_launch<double>(f, p->T, p->nlat, cols, (const double *)grid, p->d_w, p->fft.tw64,
                              (double2 *)p->H, s);
  return fft_launch<float>(f, p->T, p->nlat, cols, (const float *)grid, p->d_w, p->fft.tw32, (float2 *)p->H, s);
}

constexpr size_t kGridSmemLimit = 227 * 1024;

// Rows whose 10 padded transforms fit in shared memory take k_grid_rhs,
// longer ones k_grid_rhs_long (6 transforms, kLongThreads threads).
template <typename Rl>
static int grid_launch(const sht_plan *p, const FftArgs &f, int B, const typename cpx<Rl>::t *tw, const Rl *rowf,
                       cudaStream_t s, bool pdl) {
  typedef typename cpx<Rl>::t C;
  const size_t sm10 = 10 * (size_t)padded(f.N) * sizeof(C), sm6 = 6 * (size_t)padded(f.N) * sizeof(C);
  const bool longrows = sm10 > kGridSmemLimit;
  if (longrows && sm6 > kGridSmemLimit) return fail(PFSH_EUNSUPPORTED, "grid stage: nlon too long for this precision");
  const size_t sm = longrows ? sm6 : sm10;
  const int threads = longrows ? kLongThreads : 256;
  // centre the product rows when the last pass's leak (multiples of
  // nlon / last radix) falls inside the retained band
  const bool center = f.N / f.radix[f.npass - 1] <= p->T;
  return with_shape(f.N, [&]<typename Shape>() -> int {
    auto kern = longrows ? k_grid_rhs_long<Rl, Shape> : k_grid_rhs<Rl, Shape>;
    int rc = set_smem((const void *)kern, sm);
    if (rc) return rc;
    {
      PFSH_LAUNCH(longrows ? "k_grid_rhs_long" : "k_grid_rhs", s);
      if (pdl) {
        cudaError_t e = launch_pdl(kern, dim3(B, p->nh), dim3(threads), sm, s, f, p->T, p->nlat, B, (const C *)p->F,
                                   rowf, tw, (C *)p->H, center);
        if (e != cudaSuccess) return cuda_fail(e, "k_grid_rhs");
      } else {
        kern<<<dim3(B, p->nh), threads, sm, s>>>(f, p->T, p->nlat, B, (const C *)p->F, rowf, tw, (C *)p->H, center);
      }
    }
    PFSH_CHECK_LAUNCH("k_grid_rhs");
    return PFSH_OK;
  });
}

int grid_rhs(const sht_plan *p, int B, const swe_params &, cudaStream_t s, bool pdl) {
  FftArgs f = fft_args(p->fft);
  if (p->prec == PFSH_FP64) return grid_launch<double>(p, f, B, p->fft.tw64, p->d_rowf, s, pdl);
  return grid_launch<float>(p, f, B, p->fft.tw32, p->d_rowf32, s, pdl);
}

}  // namespace pfsh
