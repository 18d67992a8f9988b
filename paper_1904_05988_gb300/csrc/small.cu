// RHS evaluation for one or two states (the serial coarse chain of PFASST
// runs one time slice per call): three launches instead of five.
//
//   k_small_synth  per order m: the coefficient rows of eta, Phi', U, V
//                  (velocity recovery of Section 2) are computed once into
//                  shared memory, then every northern latitude accumulates
//                  the even and odd Legendre sums (K split across thread
//                  groups to shorten the dependent chain) -> F(+-mu).
//   k_grid_rhs     unchanged (fft.cu).
//   k_small_anal   per order m: one warp per degree contracts the
//                  hemispheric sums over latitude into shared memory, then
//                  the div/curl stencil assembles F_E and F_I for that order.
//
// The arithmetic is that of k_rhs_prep / legendre_* / k_rhs_assemble, in the
// plan's real type for the contractions (fp64 for FP64 plans, fp32 otherwise)
// and fp64 for the spectral parts.
#include "internal.cuh"
#include "spectral_ops.cuh"

namespace pfsh {

constexpr int kSmallMaxStates = 2;

template <typename R, int NB>
__global__ void __launch_bounds__(256) k_small_synth(int T, int nlat, int B, R ma2, R inva, double omega,
                                                     double phibar, SpecTables<R> tb, const R *__restrict__ P,
                                                     const double2 *__restrict__ state,
                                                     typename cpx<R>::t *__restrict__ F) {
  typedef typename cpx<R>::t C;
  constexpr int NC = 4 * NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = blockIdx.x, nh = nlat / 2, K = T + 2 - m, cols = 4 * B;
  const int parts = max(1, (int)blockDim.x / nh);
  const int Kc = ((K + parts - 1) / parts + 1) & ~1;          // even chunk length
  C *Xs = reinterpret_cast<C *>(smem_raw);                    // [K][cols]
  C *Ps = Xs + (size_t)K * cols;                               // [parts][nh][2][cols]
  const int nc = ncoef_of(T);
  const int base = poff(T, m) - m;
  const size_t e0 = (size_t)poff(T + 1, m);
  // 1. coefficient rows for this order
  for (int t = threadIdx.x; t < K * B; t += blockDim.x) {
    const int i = t / B, b = t - i * B;
    const double2 *Phi = state + (size_t)b * 3 * nc;
    prep_point<R>(T, m, m + i, Phi, Phi + nc, Phi + 2 * nc, base, e0 + i, tb, ma2, inva, omega, phibar,
                  Xs + (size_t)i * cols + b * 4);
  }
  __syncthreads();
  // 2. even/odd Legendre sums per latitude and K chunk
  const size_t row0 = (size_t)eoff(T, m);
  for (int t = threadIdx.x; t < nh * parts; t += blockDim.x) {
    const int j = t % nh, part = t / nh;
    const int i0 = part * Kc, i1 = min(K, i0 + Kc);
    C e[NC], o[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) e[c] = o[c] = mk<C>(0.0, 0.0);
    for (int i = i0; i < i1; i += 2) {
      const R pe = P[(row0 + i) * nh + j];
      const R po = (i + 1 < i1) ? P[(row0 + i + 1) * nh + j] : (R)0;
      const C *xe = Xs + (size_t)i * cols, *xo = xe + cols;
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < cols) {
          const C u = xe[c];
          e[c].x += pe * u.x;
          e[c].y += pe * u.y;
          if (i + 1 < i1) {
            const C v = xo[c];
            o[c].x += po * v.x;
            o[c].y += po * v.y;
          }
        }
    }
    C *ps = Ps + ((size_t)part * nh + j) * 2 * cols;
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < cols) {
        ps[c] = e[c];
        ps[cols + c] = o[c];
      }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nh * cols; t += blockDim.x) {
    const int j = t / cols, c = t - j * cols;
    C E = mk<C>(0.0, 0.0), O = mk<C>(0.0, 0.0);
    for (int part = 0; part < parts; ++part) {
      const C *ps = Ps + ((size_t)part * nh + j) * 2 * cols;
      E = E + ps[c];
      O = O + ps[cols + c];
    }
    F[((size_t)m * nlat + j) * cols + c] = E + O;
    F[((size_t)m * nlat + (nlat - 1 - j)) * cols + c] = E - O;
  }
}

template <typename R, int NB>
__global__ void __launch_bounds__(512) k_small_anal(int T, int nlat, int B, R inva, R inva2, double dinva2, double nu,
                                                    double phibar, const R *__restrict__ eps,
                                                    const R *__restrict__ P, const typename cpx<R>::t *__restrict__ H,
                                                    const double2 *__restrict__ state, double2 *__restrict__ fE,
                                                    double2 *__restrict__ fI) {
  typedef typename cpx<R>::t C;
  constexpr int NC = 5 * NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = blockIdx.x, nh = nlat / 2, K = T + 2 - m, cols = 5 * B;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  C *Ys = reinterpret_cast<C *>(smem_raw);     // [K][cols]
  const size_t row0 = (size_t)eoff(T, m);
  // 1. analysis of every degree of this order
  for (int i = warp; i < K; i += nwarps) {
    const int p = i & 1;
    const C *h = H + ((size_t)m * 2 + p) * nh * cols;
    C acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = mk<C>(0.0, 0.0);
    for (int j = lane; j < nh; j += 32) {
      const R pv = P[(row0 + i) * nh + j];
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < cols) {
          const C v = h[(size_t)j * cols + c];
          acc[c].x += pv * v.x;
          acc[c].y += pv * v.y;
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, d);
        acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, d);
      }
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (lane == c && c < cols) Ys[(size_t)i * cols + c] = acc[c];
  }
  __syncthreads();
  // 2. assembly of F_E and F_I for n = m..T
  const int nc = ncoef_of(T);
  const size_t e0 = (size_t)poff(T + 1, m);
  const int pidx0 = poff(T, m);
  for (int t = threadIdx.x; t < (T + 1 - m) * B; t += blockDim.x) {
    const int i = t / B, b = t - i * B, n = m + i;
    C cur[5], up[5], dn[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      cur[f] = Ys[(size_t)i * cols + b * 5 + f];
      up[f] = Ys[(size_t)(i + 1) * cols + b * 5 + f];
      dn[f] = i ? Ys[(size_t)(i - 1) * cols + b * 5 + f] : mk<C>(0.0, 0.0);
    }
    double2 fe[3];
    assemble_point<R, C>(m, n, cur, up, dn, i > 0, eps[e0 + i + 1], eps[e0 + i], inva, inva2, fe);
    const size_t idx = (size_t)pidx0 + i;
    double2 *oE = fE + (size_t)b * 3 * nc;
    oE[idx] = fe[0];
    oE[nc + idx] = fe[1];
    oE[2 * nc + idx] = fe[2];
    if (fI) linear_point(m, n, state + (size_t)b * 3 * nc, nc, idx, dinva2, nu, phibar, fI + (size_t)b * 3 * nc);
  }
}

template <typename R, int NB>
static int small_launch(const sht_plan *p, const double *state, double *fE, double *fI, int B, const swe_params &prm,
                        const R *P, SpecTables<R> tb, cudaStream_t s) {
  typedef typename cpx<R>::t C;
  const int nh = p->nh, K = p->T + 2;
  const int parts = std::max(1, 256 / nh);
  const size_t sm1 = ((size_t)K * 4 * B + (size_t)parts * nh * 2 * 4 * B) * sizeof(C);
  int rc = ensure_smem((const void *)k_small_synth<R, NB>, sm1);
  if (rc) return rc;
  {
    PFSH_LAUNCH("k_small_synth", s);
    k_small_synth<R, NB><<<p->T + 1, 256, sm1, s>>>(p->T, p->nlat, B, (R)(-prm.a * prm.a), (R)(1.0 / prm.a),
                                                    prm.omega, prm.phibar, tb, P, (const double2 *)state,
                                                    (C *)p->F);
  }
  PFSH_CHECK_LAUNCH("k_small_synth");
  if ((rc = grid_rhs(p, B, prm, s))) return rc;
  const size_t sm3 = (size_t)K * 5 * B * sizeof(C);
  if ((rc = ensure_smem((const void *)k_small_anal<R, NB>, sm3))) return rc;
  const double inva2 = 1.0 / (prm.a * prm.a);
  {
    PFSH_LAUNCH("k_small_anal", s);
    k_small_anal<R, NB><<<p->T + 1, 512, sm3, s>>>(p->T, p->nlat, B, (R)(1.0 / prm.a), (R)inva2, inva2, prm.nu,
                                                   prm.phibar, tb.eps, P, (const C *)p->H, (const double2 *)state,
                                                   (double2 *)fE, (double2 *)fI);
  }
  PFSH_CHECK_LAUNCH("k_small_anal");
  return PFSH_OK;
}

bool small_rhs(int B) { return B <= kSmallMaxStates; }

int rhs_small(const sht_plan *p, const double *state, double *fE, double *fI, int B, const swe_params &prm,
              cudaStream_t s) {
  const SpecTables<double> t64{p->d_eps, p->d_ilap};
  const SpecTables<float> t32{p->d_eps32, p->d_ilap32};
  if (p->prec == PFSH_FP64)
    return B == 1 ? small_launch<double, 1>(p, state, fE, fI, B, prm, p->d_P, t64, s)
                  : small_launch<double, 2>(p, state, fE, fI, B, prm, p->d_P, t64, s);
  return B == 1 ? small_launch<float, 1>(p, state, fE, fI, B, prm, p->d_P32, t32, s)
                : small_launch<float, 2>(p, state, fE, fI, B, prm, p->d_P32, t32, s);
}

}  // namespace pfsh
