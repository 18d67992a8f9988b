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

#include "internal.cuh"

namespace pfsh {

struct FftArgs {
  int N, npass;
  int radix[kMaxPasses];
};

static FftArgs fft_args(const FftPlan &f) {
  FftArgs a;
  a.N = f.N;
  a.npass = f.npass;
  for (int i = 0; i < kMaxPasses; ++i) a.radix[i] = i < f.npass ? f.radix[i] : 1;
  return a;
}

template <typename C> __device__ __forceinline__ C twiddle(const C *tw, int e, bool inv) {
  C w = tw[e];
  if (inv) w.y = -w.y;
  return w;
}

// nfft transforms of length N stored back to back in `a`; `b` is scratch of
// the same size.  Returns the buffer that holds the result.  Must be called
// by every thread of the block.
template <typename C>
__device__ C *fft_smem(C *a, C *b, int nfft, const FftArgs &f, const C *__restrict__ tw, bool inv) {
  const int N = f.N;
  int Ns = 1;
  for (int p = 0; p < f.npass; ++p) {
    const int R = f.radix[p];
    const int NR = N / R;
    const int stride = N / (Ns * R);
    const int total = nfft * NR;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int fi = t / NR;
      const int j = t - fi * NR;
      const C *x = a + fi * N;
      C *y = b + fi * N;
      const int k = j % Ns;
      const int idx = (j / Ns) * Ns * R + k;
      if (R == 4) {
        C v0 = x[j];
        C v1 = cmul(x[j + NR], twiddle(tw, k * stride, inv));
        C v2 = cmul(x[j + 2 * NR], twiddle(tw, 2 * k * stride, inv));
        C v3 = cmul(x[j + 3 * NR], twiddle(tw, 3 * k * stride, inv));
        C s02 = v0 + v2, d02 = v0 - v2, s13 = v1 + v3, d13 = v1 - v3;
        C rot = times_i(d13);  // i (v1 - v3)
        y[idx] = s02 + s13;
        y[idx + 2 * Ns] = s02 - s13;
        if (!inv) {
          y[idx + Ns] = d02 - rot;
          y[idx + 3 * Ns] = d02 + rot;
        } else {
          y[idx + Ns] = d02 + rot;
          y[idx + 3 * Ns] = d02 - rot;
        }
      } else if (R == 2) {
        C v0 = x[j];
        C v1 = cmul(x[j + NR], twiddle(tw, k * stride, inv));
        y[idx] = v0 + v1;
        y[idx + Ns] = v0 - v1;
      } else if (R == 3) {
        C v0 = x[j];
        C v1 = cmul(x[j + NR], twiddle(tw, k * stride, inv));
        C v2 = cmul(x[j + 2 * NR], twiddle(tw, 2 * k * stride, inv));
        typedef decltype(v0.x) Rt;
        const Rt c = (Rt)-0.5;
        const Rt s = inv ? (Rt)0.86602540378443864676 : (Rt)-0.86602540378443864676;
        C t = v1 + v2, u = v1 - v2;
        C base = v0 + c * t;
        C su = times_i(s * u);
        y[idx] = v0 + t;
        y[idx + Ns] = base + su;
        y[idx + 2 * Ns] = base - su;
      } else {
        // direct DFT of length R (5 and odd primes up to 61)
        for (int q = 0; q < R; ++q) {
          C acc = mk<C>(0.0, 0.0);
          for (int r = 0; r < R; ++r) {
            C v = x[j + r * NR];
            if (r) v = cmul(v, twiddle(tw, k * r * stride, inv));
            const int e = (r * q) % R;
            acc = acc + (e ? cmul(v, twiddle(tw, e * NR, inv)) : v);
          }
          y[idx + q * Ns] = acc;
        }
      }
    }
    __syncthreads();
    C *tmp = a;
    a = b;
    b = tmp;
    Ns *= R;
  }
  return a;
}

// ---------------------------------------------------------------------------
// inverse: F[m][lat][col] -> grid[col][lat][lon]
// ---------------------------------------------------------------------------
template <typename Rl>
__global__ void k_ifft_rows(FftArgs f, int T, int nlat, int cols, const typename cpx<Rl>::t *__restrict__ F,
                            const typename cpx<Rl>::t *__restrict__ tw, Rl *__restrict__ grid) {
  typedef typename cpx<Rl>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *a = reinterpret_cast<C *>(smem_raw);
  C *b = a + f.N;
  const int j = blockIdx.x, col = blockIdx.y, js = nlat - 1 - j;
  const int N = f.N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) a[k] = mk<C>(0.0, 0.0);
  __syncthreads();
  for (int m = threadIdx.x; m <= T; m += blockDim.x) {
    C fn = F[((size_t)m * nlat + j) * cols + col];
    C fs = F[((size_t)m * nlat + js) * cols + col];
    if (m == 0) {
      a[0] = mk<C>(fn.x, fs.x);
    } else {
      a[m] = mk<C>(fn.x - fs.y, fn.y + fs.x);
      a[N - m] = mk<C>(fn.x + fs.y, -fn.y + fs.x);
    }
  }
  __syncthreads();
  C *r = fft_smem<C>(a, b, 1, f, tw, true);
  Rl *gn = grid + ((size_t)col * nlat + j) * N;
  Rl *gs = grid + ((size_t)col * nlat + js) * N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    C z = r[k];
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
    C zm = Z[m];
    C zc = cconj(Z[m == 0 ? 0 : N - m]);
    C gn = half * (zm + zc);              // north spectrum
    C gs = half * times_i(zc - zm);       // south spectrum: (zm - zc) / (2i)
    C he = wj * (gn + gs), ho = wj * (gn - gs);
    H[(((size_t)m * 2 + 0) * nh + j) * cols + col] = he;
    H[(((size_t)m * 2 + 1) * nh + j) * cols + col] = ho;
  }
}

template <typename Rl>
__global__ void k_fft_rows(FftArgs f, int T, int nlat, int cols, const Rl *__restrict__ grid,
                           const double *__restrict__ w, const typename cpx<Rl>::t *__restrict__ tw,
                           typename cpx<Rl>::t *__restrict__ H) {
  typedef typename cpx<Rl>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *a = reinterpret_cast<C *>(smem_raw);
  C *b = a + f.N;
  const int j = blockIdx.x, col = blockIdx.y, js = nlat - 1 - j, N = f.N;
  const Rl *gn = grid + ((size_t)col * nlat + j) * N;
  const Rl *gs = grid + ((size_t)col * nlat + js) * N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) a[k] = mk<C>(gn[k], gs[k]);
  __syncthreads();
  C *r = fft_smem<C>(a, b, 1, f, tw, false);
  unpack_write<C, Rl>(r, N, T, j, nlat / 2, cols, col, (Rl)w[j], H);
}

// ---------------------------------------------------------------------------
// RHS grid stage: 4 spectra (eta, Phi', U, V) per state -> 5 products
//   A1 = eta U/(1-mu^2), B1 = eta V/(1-mu^2), A2 = Phi' U/(1-mu^2),
//   B2 = Phi' V/(1-mu^2), E = (U^2+V^2)/(2(1-mu^2))
// F columns: b*4 + f ; H columns: b*5 + f
// ---------------------------------------------------------------------------
template <typename Rl>
__global__ void k_grid_rhs(FftArgs f, int T, int nlat, int B, const typename cpx<Rl>::t *__restrict__ F,
                           const double *__restrict__ mu, const double *__restrict__ w,
                           const typename cpx<Rl>::t *__restrict__ tw, typename cpx<Rl>::t *__restrict__ H) {
  typedef typename cpx<Rl>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = f.N;
  C *A = reinterpret_cast<C *>(smem_raw);  // 5N
  C *Bf = A + 5 * N;                        // 5N
  const int j = blockIdx.x, b = blockIdx.y, js = nlat - 1 - j;
  const int colsF = 4 * B, colsH = 5 * B;
  for (int k = threadIdx.x; k < 4 * N; k += blockDim.x) A[k] = mk<C>(0.0, 0.0);
  __syncthreads();
  for (int t = threadIdx.x; t < 4 * (T + 1); t += blockDim.x) {
    const int fld = t / (T + 1), m = t - fld * (T + 1);
    C fn = F[((size_t)m * nlat + j) * colsF + b * 4 + fld];
    C fs = F[((size_t)m * nlat + js) * colsF + b * 4 + fld];
    C *z = A + fld * N;
    if (m == 0) {
      z[0] = mk<C>(fn.x, fs.x);
    } else {
      z[m] = mk<C>(fn.x - fs.y, fn.y + fs.x);
      z[N - m] = mk<C>(fn.x + fs.y, -fn.y + fs.x);
    }
  }
  __syncthreads();
  C *g = fft_smem<C>(A, Bf, 4, f, tw, true);
  C *o = (g == A) ? Bf : A;
  const double x = mu[j];
  const Rl inv = (Rl)(1.0 / ((1.0 - x) * (1.0 + x)));
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    C eta = g[k], php = g[N + k], U = g[2 * N + k], V = g[3 * N + k];
    Rl etaU_n = eta.x * U.x * inv, etaU_s = eta.y * U.y * inv;
    Rl etaV_n = eta.x * V.x * inv, etaV_s = eta.y * V.y * inv;
    o[k] = mk<C>(etaU_n, etaU_s);
    o[N + k] = mk<C>(etaV_n, etaV_s);
    o[2 * N + k] = mk<C>(php.x * U.x * inv, php.y * U.y * inv);
    o[3 * N + k] = mk<C>(php.x * V.x * inv, php.y * V.y * inv);
    const Rl h = (Rl)0.5 * inv;
    o[4 * N + k] = mk<C>((U.x * U.x + V.x * V.x) * h, (U.y * U.y + V.y * V.y) * h);
  }
  __syncthreads();
  C *Z = fft_smem<C>(o, g, 5, f, tw, false);
  const Rl half = (Rl)0.5 / (Rl)N;
  const Rl wj = (Rl)w[j];
  const int nh = nlat / 2;
  for (int t = threadIdx.x; t < 5 * (T + 1); t += blockDim.x) {
    const int fld = t / (T + 1), m = t - fld * (T + 1);
    const C *z = Z + fld * N;
    C zm = z[m];
    C zc = cconj(z[m == 0 ? 0 : N - m]);
    C gn = half * (zm + zc);
    C gs = half * times_i(zc - zm);
    C he = wj * (gn + gs), ho = wj * (gn - gs);
    H[(((size_t)m * 2 + 0) * nh + j) * colsH + b * 5 + fld] = he;
    H[(((size_t)m * 2 + 1) * nh + j) * colsH + b * 5 + fld] = ho;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int set_smem(const void *fn, size_t bytes) {
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
  }
  return PFSH_OK;
}

int ifft_rows(const sht_plan *p, int cols, void *grid, cudaStream_t s) {
  FftArgs f = fft_args(p->fft);
  dim3 g(p->nh, cols);
  if (p->prec == PFSH_FP64) {
    size_t sm = 2 * (size_t)f.N * sizeof(double2);
    int rc = set_smem((const void *)k_ifft_rows<double>, sm);
    if (rc) return rc;
    {
      PFSH_LAUNCH("k_ifft_rows", s);
      k_ifft_rows<double><<<g, 256, sm, s>>>(f, p->T, p->nlat, cols, (const double2 *)p->F, p->fft.tw64,
                                             (double *)grid);
    }
  } else {
    size_t sm = 2 * (size_t)f.N * sizeof(float2);
    int rc = set_smem((const void *)k_ifft_rows<float>, sm);
    if (rc) return rc;
    {
      PFSH_LAUNCH("k_ifft_rows", s);
      k_ifft_rows<float><<<g, 256, sm, s>>>(f, p->T, p->nlat, cols, (const float2 *)p->F, p->fft.tw32,
                                            (float *)grid);
    }
  }
  PFSH_CHECK_LAUNCH("k_ifft_rows");
  return PFSH_OK;
}

// Inverse longitude transform of F[m][lat][cols] (complex fp64) into
// grid[cols][lat][lon] with caller-supplied twiddles and radix list; used by
// the allocation-free synthesis entry point.
int ifft_rows_f64_raw(int N, int npass, const int *radix, int T, int nlat, int cols, const double2 *F,
                      const double2 *tw, double *grid, cudaStream_t s) {
  FftArgs f;
  f.N = N;
  f.npass = npass;
  for (int i = 0; i < kMaxPasses; ++i) f.radix[i] = i < npass ? radix[i] : 1;
  const size_t sm = 2 * (size_t)N * sizeof(double2);
  int rc = set_smem((const void *)k_ifft_rows<double>, sm);
  if (rc) return rc;
  {
    PFSH_LAUNCH("k_ifft_rows", s);
    k_ifft_rows<double><<<dim3(nlat / 2, cols), 256, sm, s>>>(f, T, nlat, cols, F, tw, grid);
  }
  PFSH_CHECK_LAUNCH("k_ifft_rows");
  return PFSH_OK;
}

int fft_rows(const sht_plan *p, int cols, const void *grid, cudaStream_t s) {
  FftArgs f = fft_args(p->fft);
  dim3 g(p->nh, cols);
  if (p->prec == PFSH_FP64) {
    size_t sm = 2 * (size_t)f.N * sizeof(double2);
    int rc = set_smem((const void *)k_fft_rows<double>, sm);
    if (rc) return rc;
    {
      PFSH_LAUNCH("k_fft_rows", s);
      k_fft_rows<double><<<g, 256, sm, s>>>(f, p->T, p->nlat, cols, (const double *)grid, p->d_w, p->fft.tw64,
                                            (double2 *)p->H);
    }
  } else {
    size_t sm = 2 * (size_t)f.N * sizeof(float2);
    int rc = set_smem((const void *)k_fft_rows<float>, sm);
    if (rc) return rc;
    {
      PFSH_LAUNCH("k_fft_rows", s);
      k_fft_rows<float><<<g, 256, sm, s>>>(f, p->T, p->nlat, cols, (const float *)grid, p->d_w, p->fft.tw32,
                                           (float2 *)p->H);
    }
  }
  PFSH_CHECK_LAUNCH("k_fft_rows");
  return PFSH_OK;
}

int grid_rhs(const sht_plan *p, int B, const swe_params &, cudaStream_t s) {
  FftArgs f = fft_args(p->fft);
  dim3 g(p->nh, B);
  if (p->prec == PFSH_FP64) {
    size_t sm = 10 * (size_t)f.N * sizeof(double2);
    int rc = set_smem((const void *)k_grid_rhs<double>, sm);
    if (rc) return rc;
    {
      PFSH_LAUNCH("k_grid_rhs", s);
      k_grid_rhs<double><<<g, 256, sm, s>>>(f, p->T, p->nlat, B, (const double2 *)p->F, p->d_mu, p->d_w,
                                            p->fft.tw64, (double2 *)p->H);
    }
  } else {
    size_t sm = 10 * (size_t)f.N * sizeof(float2);
    int rc = set_smem((const void *)k_grid_rhs<float>, sm);
    if (rc) return rc;
    {
      PFSH_LAUNCH("k_grid_rhs", s);
      k_grid_rhs<float><<<g, 256, sm, s>>>(f, p->T, p->nlat, B, (const float2 *)p->F, p->d_mu, p->d_w,
                                           p->fft.tw32, (float2 *)p->H);
    }
  }
  PFSH_CHECK_LAUNCH("k_grid_rhs");
  return PFSH_OK;
}

}  // namespace pfsh
