// Legendre contractions per order m on CUDA cores (the discrete Legendre
// transform of Section 3): FP64 for the plain FP64 path, FP32 for PFSH_FP32.
//
// Synthesis, for every m and complex column c (a field of a batch entry):
//   S_p(mu_j) = sum_{n-m = p mod 2} P_n^m(mu_j) X_n^m[c],  p = 0, 1,
//   F_m(+mu_j) = S_0 + S_1,   F_m(-mu_j) = S_0 - S_1,
// using P_n^m(-mu) = (-1)^{n-m} P_n^m(mu), so only northern rows of the
// table are stored.  Analysis reverses it with the hemispheric sums H_p
// (already weighted by w_j) produced by the longitude stage:
//   Y_n^m[c] = sum_{j north} P_n^m(mu_j) H_{(n-m) mod 2}[m][j][c].
// Both are shared-memory tiled GEMMs on CUDA cores, templated on the real
// type R of the table, the operands and the accumulators.
#include "internal.cuh"

namespace pfsh {

constexpr int TJ = 32;  // latitude / degree tile
constexpr int TC = 32;  // complex-column tile
constexpr int TK = 16;  // contraction chunk

// grid: (ceil(nh/TJ), ceil(cols/TC), T+1); block 256 = 16 (j) x 16 (c), each
// thread 2 latitudes x 2 columns x 2 parities.
template <typename R>
__global__ void __launch_bounds__(256) k_synth_simt(int T, int nlat, int cols, const R *__restrict__ P,
                                                    const typename cpx<R>::t *__restrict__ X,
                                                    typename cpx<R>::t *__restrict__ F) {
  typedef typename cpx<R>::t C;
  __shared__ R Ps[TK][TJ];
  __shared__ C Xs[TK][TC];
  const int m = blockIdx.z;
  const int nh = nlat / 2;
  const int j0 = blockIdx.x * TJ, c0 = blockIdx.y * TC;
  const int tj = threadIdx.x / 16, tc = threadIdx.x % 16;
  const int K = T + 2 - m;
  const size_t row0 = (size_t)eoff(T, m);
  C acc[2][2][2];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) acc[p][a][b] = mk<C>(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int t = threadIdx.x; t < TK * TJ; t += 256) {
      int r = t / TJ, jj = t % TJ;
      int j = j0 + jj;
      Ps[r][jj] = (k0 + r < K && j < nh) ? P[(row0 + k0 + r) * nh + j] : (R)0;
    }
    for (int t = threadIdx.x; t < TK * TC; t += 256) {
      int r = t / TC, cc = t % TC;
      int c = c0 + cc;
      Xs[r][cc] = (k0 + r < K && c < cols) ? X[(row0 + k0 + r) * cols + c] : mk<C>(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TK; r += 2) {
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        R pa = Ps[r + p][tj * 2], pb = Ps[r + p][tj * 2 + 1];
        C xa = Xs[r + p][tc * 2], xb = Xs[r + p][tc * 2 + 1];
        acc[p][0][0].x = fma(pa, xa.x, acc[p][0][0].x); acc[p][0][0].y = fma(pa, xa.y, acc[p][0][0].y);
        acc[p][0][1].x = fma(pa, xb.x, acc[p][0][1].x); acc[p][0][1].y = fma(pa, xb.y, acc[p][0][1].y);
        acc[p][1][0].x = fma(pb, xa.x, acc[p][1][0].x); acc[p][1][0].y = fma(pb, xa.y, acc[p][1][0].y);
        acc[p][1][1].x = fma(pb, xb.x, acc[p][1][1].x); acc[p][1][1].y = fma(pb, xb.y, acc[p][1][1].y);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    int j = j0 + tj * 2 + a;
    if (j >= nh) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int c = c0 + tc * 2 + b;
      if (c >= cols) continue;
      C s0 = acc[0][a][b], s1 = acc[1][a][b];
      F[((size_t)m * nlat + j) * cols + c] = s0 + s1;
      F[((size_t)m * nlat + (nlat - 1 - j)) * cols + c] = s0 - s1;
    }
  }
}

// grid: (ceil((T+2)/TJ), ceil(cols/TC), T+1); block 256 = 16 (n pairs) x 16 (c).
// Thread (tn, tc) owns degrees n-m = 2*tn', 2*tn'+1 within the tile (one even,
// one odd) and 2 columns.
template <typename R>
__global__ void __launch_bounds__(256) k_anal_simt(int T, int nlat, int cols, const R *__restrict__ P,
                                                   const typename cpx<R>::t *__restrict__ H,
                                                   typename cpx<R>::t *__restrict__ Y) {
  typedef typename cpx<R>::t C;
  __shared__ R Ps[TJ][TK + 1];       // [degree in tile][lat chunk]
  __shared__ C Hs[2][TK][TC];        // [parity][lat chunk][col]
  const int m = blockIdx.z;
  const int K = T + 2 - m;
  const int i0 = blockIdx.x * TJ;
  if (i0 >= K) return;
  const int nh = nlat / 2;
  const int c0 = blockIdx.y * TC;
  const int tn = threadIdx.x / 16, tc = threadIdx.x % 16;
  const size_t row0 = (size_t)eoff(T, m);
  C acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = mk<C>(0.0, 0.0);
  for (int q0 = 0; q0 < nh; q0 += TK) {
    for (int t = threadIdx.x; t < TJ * TK; t += 256) {
      int r = t / TK, q = t % TK;
      int i = i0 + r, j = q0 + q;
      Ps[r][q] = (i < K && j < nh) ? P[(row0 + i) * nh + j] : (R)0;
    }
    for (int t = threadIdx.x; t < 2 * TK * TC; t += 256) {
      int p = t / (TK * TC), rem = t % (TK * TC);
      int q = rem / TC, cc = rem % TC;
      int j = q0 + q, c = c0 + cc;
      Hs[p][q][cc] = (j < nh && c < cols) ? H[(((size_t)m * 2 + p) * nh + j) * cols + c] : mk<C>(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < TK; ++q) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int r = tn * 2 + a;          // local degree index; parity = a (i0 even)
        R pv = Ps[r][q];
        C ha = Hs[a][q][tc * 2], hb = Hs[a][q][tc * 2 + 1];
        acc[a][0].x = fma(pv, ha.x, acc[a][0].x); acc[a][0].y = fma(pv, ha.y, acc[a][0].y);
        acc[a][1].x = fma(pv, hb.x, acc[a][1].x); acc[a][1].y = fma(pv, hb.y, acc[a][1].y);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    int i = i0 + tn * 2 + a;
    if (i >= K) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int c = c0 + tc * 2 + b;
      if (c < cols) Y[(row0 + i) * cols + c] = acc[a][b];
    }
  }
}

// ---------------------------------------------------------------------------
// small batches (the serial coarse chain runs one time slice per call)
// ---------------------------------------------------------------------------
// Synthesis: one thread per northern latitude of one order m, all (<= NC)
// columns in registers, no shared memory and no barriers: the table row is
// read coalesced across threads, the coefficient row is a broadcast.
template <typename R, int NC>
__global__ void __launch_bounds__(64) k_synth_small(int T, int nlat, int cols, const R *__restrict__ P,
                                                    const typename cpx<R>::t *__restrict__ X,
                                                    typename cpx<R>::t *__restrict__ F) {
  typedef typename cpx<R>::t C;
  const int m = blockIdx.y;
  const int nh = nlat / 2;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nh) return;
  const int K = T + 2 - m;
  const size_t row0 = (size_t)eoff(T, m);
  C e[NC], o[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) e[c] = o[c] = mk<C>(0.0, 0.0);
#pragma unroll 4
  for (int i = 0; i < K; i += 2) {
    const R pe = P[(row0 + i) * nh + j];
    const R po = (i + 1 < K) ? P[(row0 + i + 1) * nh + j] : (R)0;
    const C *xe = X + (row0 + i) * cols;
    const C *xo = X + (row0 + i + 1) * cols;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (c < cols) {
        const C a = xe[c];
        e[c].x += pe * a.x;
        e[c].y += pe * a.y;
        if (i + 1 < K) {
          const C b = xo[c];
          o[c].x += po * b.x;
          o[c].y += po * b.y;
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (c < cols) {
      F[((size_t)m * nlat + j) * cols + c] = e[c] + o[c];
      F[((size_t)m * nlat + (nlat - 1 - j)) * cols + c] = e[c] - o[c];
    }
}

// Analysis: one warp per degree of one order m; lanes stride over the
// latitudes and the partial sums of every column are reduced by shuffles.
template <typename R, int NC>
__global__ void __launch_bounds__(128) k_anal_small(int T, int nlat, int cols, const R *__restrict__ P,
                                                    const typename cpx<R>::t *__restrict__ H,
                                                    typename cpx<R>::t *__restrict__ Y) {
  typedef typename cpx<R>::t C;
  const int m = blockIdx.y;
  const int i = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int K = T + 2 - m;
  if (i >= K) return;
  const int nh = nlat / 2, p = i & 1;
  const size_t row = (size_t)eoff(T, m) + i;
  const C *h = H + ((size_t)m * 2 + p) * nh * cols;
  C acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = mk<C>(0.0, 0.0);
  for (int j = lane; j < nh; j += 32) {
    const R pv = P[row * nh + j];
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < cols) {
        const C v = h[(size_t)j * cols + c];
        acc[c].x += pv * v.x;
        acc[c].y += pv * v.y;
      }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, d);
      acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, d);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < cols) Y[row * cols + c] = acc[c];
  }
}

constexpr int kSmallSynthCols = 8;    // complex columns (2 states of 4 fields)
constexpr int kSmallAnalCols = 10;    // 2 states of 5 fields

int synth_small(const sht_plan *p, int cols, cudaStream_t s) {
  dim3 g((p->nh + 63) / 64, p->T + 1);
  if (p->prec == PFSH_FP64) {
    PFSH_LAUNCH("k_synth_small_f64", s);
    k_synth_small<double, kSmallSynthCols><<<g, 64, 0, s>>>(p->T, p->nlat, cols, p->d_P, (const double2 *)p->X,
                                                             (double2 *)p->F);
  } else {
    PFSH_LAUNCH("k_synth_small_f32", s);
    k_synth_small<float, kSmallSynthCols><<<g, 64, 0, s>>>(p->T, p->nlat, cols, p->d_P32, (const float2 *)p->X,
                                                            (float2 *)p->F);
  }
  PFSH_CHECK_LAUNCH("k_synth_small");
  return PFSH_OK;
}

int analysis_small(const sht_plan *p, int cols, cudaStream_t s) {
  dim3 g((p->T + 2 + 3) / 4, p->T + 1);
  if (p->prec == PFSH_FP64) {
    PFSH_LAUNCH("k_anal_small_f64", s);
    k_anal_small<double, kSmallAnalCols><<<g, 128, 0, s>>>(p->T, p->nlat, cols, p->d_P, (const double2 *)p->H,
                                                            (double2 *)p->Y);
  } else {
    PFSH_LAUNCH("k_anal_small_f32", s);
    k_anal_small<float, kSmallAnalCols><<<g, 128, 0, s>>>(p->T, p->nlat, cols, p->d_P32, (const float2 *)p->H,
                                                           (float2 *)p->Y);
  }
  PFSH_CHECK_LAUNCH("k_anal_small");
  return PFSH_OK;
}

bool small_synth(int cols) { return cols <= kSmallSynthCols; }
bool small_analysis(int cols) { return cols <= kSmallAnalCols; }

int synth_simt(const sht_plan *p, int cols, cudaStream_t s) {
  dim3 g((p->nh + TJ - 1) / TJ, (cols + TC - 1) / TC, p->T + 1);
  if (p->prec == PFSH_FP64) {
    PFSH_LAUNCH("k_synth_f64", s);
    k_synth_simt<double><<<g, 256, 0, s>>>(p->T, p->nlat, cols, p->d_P, (const double2 *)p->X, (double2 *)p->F);
  } else {
    PFSH_LAUNCH("k_synth_f32", s);
    k_synth_simt<float><<<g, 256, 0, s>>>(p->T, p->nlat, cols, p->d_P32, (const float2 *)p->X, (float2 *)p->F);
  }
  PFSH_CHECK_LAUNCH("k_synth_simt");
  return PFSH_OK;
}

int analysis_simt(const sht_plan *p, int cols, cudaStream_t s) {
  dim3 g((p->T + 2 + TJ - 1) / TJ, (cols + TC - 1) / TC, p->T + 1);
  if (p->prec == PFSH_FP64) {
    PFSH_LAUNCH("k_anal_f64", s);
    k_anal_simt<double><<<g, 256, 0, s>>>(p->T, p->nlat, cols, p->d_P, (const double2 *)p->H, (double2 *)p->Y);
  } else {
    PFSH_LAUNCH("k_anal_f32", s);
    k_anal_simt<float><<<g, 256, 0, s>>>(p->T, p->nlat, cols, p->d_P32, (const float2 *)p->H, (float2 *)p->Y);
  }
  PFSH_CHECK_LAUNCH("k_anal_simt");
  return PFSH_OK;
}

}  // namespace pfsh
