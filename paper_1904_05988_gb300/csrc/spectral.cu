// Spectral-space FP64 kernels: velocity recovery and assembly of the
// nonlinear term (Section 2), the implicit solve (Section 5.4), the IMEX-SDC
// node update (Section 5.1.1) and the FAS / space-time transfer operators
// (Sections 5.1.2 and 5.3).  All are element-wise over triangular spectral
// arrays and bound by HBM traffic or FP64 issue rate.
#include "internal.cuh"
#include "spectral_ops.cuh"

namespace pfsh {

// order m of packed index idx in a degree-T triangle (largest m with poff <= idx)
__device__ __forceinline__ int tri_m(int idx, int T) {
  const float b = 2.f * T + 3.f;
  int m = (int)((b - sqrtf(fmaxf(b * b - 8.f * idx, 0.f))) * 0.5f);
  m = max(0, min(m, T));
  while (m > 0 && poff(T, m) > idx) --m;
  while (m < T && poff(T, m + 1) <= idx) ++m;
  return m;
}

__device__ __forceinline__ double eps_nm(int n, int m) {
  if (n <= m) return 0.0;
  return sqrt(((double)n * n - (double)m * m) / (4.0 * (double)n * n - 1.0));
}

// ---------------------------------------------------------------------------
// plain transforms: spec [b][ncoef] <-> X/Y [ext row][b]
//
// The kernels between a state-major array and a row-major X/Y take blocks
// (state b, chunk of 256 rows): the blocks of all states that share a chunk of
// rows run side by side, so each row of X/Y is read or written whole while it
// is in L2 (at T1279 the arrays are larger than L2).
// ---------------------------------------------------------------------------
template <typename CX>
__global__ void k_spec_to_X(int T, int ne, int batch, const double2 *__restrict__ spec, CX *__restrict__ X) {
  int idx = blockIdx.y * blockDim.x + threadIdx.x;
  int b = blockIdx.x;
  if (idx >= ne) return;
  const int m = tri_m(idx, T + 1);  // extended triangle == packed triangle of degree T+1
  const int n = m + (idx - poff(T + 1, m));
  double2 v = make_double2(0.0, 0.0);
  if (n <= T) {
    v = spec[(size_t)b * ncoef_of(T) + poff(T, m) + (n - m)];
    if (m == 0) v.y = 0.0;
  }
  X[(size_t)idx * batch + b] = mk<CX>(v.x, v.y);
}

template <typename CY>
__global__ void k_Y_to_spec(int T, int batch, const CY *__restrict__ Y, double2 *__restrict__ spec) {
  int idx = blockIdx.y * blockDim.x + threadIdx.x;
  int b = blockIdx.x;
  const int nc = ncoef_of(T);
  if (idx >= nc) return;
  const int m = tri_m(idx, T);
  const int n = m + (idx - poff(T, m));
  const CY y = Y[(size_t)(poff(T + 1, m) + (n - m)) * batch + b];
  double2 v = make_double2(y.x, m == 0 ? 0.0 : y.y);
  spec[(size_t)b * nc + idx] = v;
}

int spec_to_X(const sht_plan *p, const double *spec, int batch, cudaStream_t s) {
  dim3 g(batch, (p->ne + 255) / 256);
  {
    PFSH_LAUNCH("k_spec_to_X", s);
    if (p->prec == PFSH_FP64)
      k_spec_to_X<double2><<<g, 256, 0, s>>>(p->T, p->ne, batch, (const double2 *)spec, (double2 *)p->X);
    else
      k_spec_to_X<float2><<<g, 256, 0, s>>>(p->T, p->ne, batch, (const double2 *)spec, (float2 *)p->X);
  }
  PFSH_CHECK_LAUNCH("k_spec_to_X");
  return PFSH_OK;
}

int Y_to_spec(const sht_plan *p, double *spec, int batch, cudaStream_t s) {
  dim3 g(batch, (p->ncoef + 255) / 256);
  {
    PFSH_LAUNCH("k_Y_to_spec", s);
    if (p->prec == PFSH_FP64)
      k_Y_to_spec<double2><<<g, 256, 0, s>>>(p->T, batch, (const double2 *)p->Y, (double2 *)spec);
    else
      k_Y_to_spec<float2><<<g, 256, 0, s>>>(p->T, batch, (const float2 *)p->Y, (double2 *)spec);
  }
  PFSH_CHECK_LAUNCH("k_Y_to_spec");
  return PFSH_OK;
}

// ---------------------------------------------------------------------------
// RHS prep: state [b][3][ncoef] -> X[ext row][b*4 + f], f = eta, Phi', U, V
//   eta  = zeta + 2 Omega mu           (mu = P_1^0 / sqrt(3/2))
//   Phi' = Phi - Phibar                 (1 = sqrt(2) P_0^0)
//   psi_n = -a^2 zeta_n / (n(n+1)), chi_n likewise (n >= 1; 0 at n = 0)
//   U_n = [(n-1) eps_n psi_{n-1} - (n+2) eps_{n+1} psi_{n+1} + i m chi_n] / a
//   V_n = [i m psi_n - (n-1) eps_n chi_{n-1} + (n+2) eps_{n+1} chi_{n+1}] / a
// ---------------------------------------------------------------------------
template <typename M>
__global__ void k_rhs_prep(int T, int ne, int B, int cnt, size_t nstride, M ma2, M inva, double omega,
                           double phibar, SpecTables<M> tb, const double2 *__restrict__ state,
                           typename cpx<M>::t *__restrict__ X) {
  typedef typename cpx<M>::t C;
  int idx = blockIdx.y * blockDim.x + threadIdx.x;
  int b = blockIdx.x;
  if (idx >= ne) return;
  const int nc = ncoef_of(T);
  const int m = tri_m(idx, T + 1);
  const int n = m + (idx - poff(T + 1, m));
  const double2 *Phi = state + (size_t)(b / cnt) * nstride + (size_t)(b % cnt) * 3 * nc;
  C out[4];
  prep_point<M>(T, m, n, Phi, Phi + nc, Phi + 2 * nc, poff(T, m) - m, (size_t)idx, tb, ma2, inva, omega, phibar, out);
  C *row = X + (size_t)idx * (4 * B) + b * 4;
  row[0] = out[0];
  row[1] = out[1];
  row[2] = out[2];
  row[3] = out[3];
}

int rhs_prep(const sht_plan *p, const double *state, int B, const swe_params &prm, cudaStream_t s, int cnt,
             size_t nstride) {
  if (cnt <= 0) cnt = B;
  nstride /= 2;   // doubles -> complex elements
  dim3 g(B, (p->ne + 255) / 256);
  {
    PFSH_LAUNCH("k_rhs_prep", s);
    if (p->prec == PFSH_FP64)
      k_rhs_prep<double><<<g, 256, 0, s>>>(p->T, p->ne, B, cnt, nstride, -prm.a * prm.a, 1.0 / prm.a, omega_explicit(prm),
                                           prm.phibar,
                                           SpecTables<double>{p->d_eps, p->d_ilap}, (const double2 *)state,
                                           (double2 *)p->X);
    else
      k_rhs_prep<float><<<g, 256, 0, s>>>(p->T, p->ne, B, cnt, nstride, (float)(-prm.a * prm.a), (float)(1.0 / prm.a),
                                          omega_explicit(prm), prm.phibar, SpecTables<float>{p->d_eps32, p->d_ilap32},
                                          (const double2 *)state, (float2 *)p->X);
  }
  PFSH_CHECK_LAUNCH("k_rhs_prep");
  return PFSH_OK;
}

// ---------------------------------------------------------------------------
// RHS assembly: Y[ext row][b*5 + f] (f = A1, B1, A2, B2, E analysed with the
// 1/(1-mu^2) factor) -> F_E, and F_I from the state:
//   div_n  = [i m A_n + n eps_{n+1} B_{n+1} - (n+1) eps_n B_{n-1}] / a
//   curl_n = [i m B_n - n eps_{n+1} A_{n+1} + (n+1) eps_n A_{n-1}] / a
//   F_E = [-div(A2,B2), -div(A1,B1), curl(A1,B1) + n(n+1)/a^2 E]
//   F_I = [-Phibar delta - nu k Phi, -nu k zeta, k Phi - nu k delta], k = n(n+1)/a^2
// ---------------------------------------------------------------------------
template <typename M>
__global__ void k_rhs_assemble(int T, int B, int cnt, size_t nstride, M inva, M inva2, double dinva2, double nu,
                               double phibar,
                               CorArgs cor, const M *__restrict__ eps, const typename cpx<M>::t *__restrict__ Y,
                               const double2 *__restrict__ state, double2 *__restrict__ fE,
                               double2 *__restrict__ fI) {
  typedef typename cpx<M>::t C;
  int idx = blockIdx.y * blockDim.x + threadIdx.x;
  int b = blockIdx.x;
  const int nc = ncoef_of(T);
  if (idx >= nc) return;
  const int m = tri_m(idx, T);
  const int n = m + (idx - poff(T, m));
  const int cols = 5 * B;
  const size_t r0 = (size_t)(poff(T + 1, m) + (n - m));
  C cur[5], up[5], dn[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    cur[f] = Y[r0 * cols + b * 5 + f];
    up[f] = Y[(r0 + 1) * cols + b * 5 + f];
    dn[f] = n > m ? Y[(r0 - 1) * cols + b * 5 + f] : mk<C>(0.0, 0.0);
  }
  double2 fe[3];
  assemble_point<M, C>(m, n, cur, up, dn, n > m, eps[r0 + 1], eps[r0], inva, inva2, fe);
  const size_t sb = (size_t)(b / cnt) * nstride + (size_t)(b % cnt) * 3 * nc;   // state b of the batch
  double2 *oE = fE + sb;
  oE[idx] = fe[0];
  oE[nc + idx] = fe[1];
  oE[2 * nc + idx] = fe[2];
  if (fI) linear_point(m, n, T, state + sb, nc, idx, dinva2, nu, phibar, cor, fI + sb);
}

int rhs_assemble(const sht_plan *p, const double *state, double *fE, double *fI, int B, const swe_params &prm,
                 CorArgs cor, cudaStream_t s, int cnt, size_t nstride) {
  if (cnt <= 0) cnt = B;
  nstride /= 2;   // doubles -> complex elements
  dim3 g(B, (p->ncoef + 255) / 256);
  const double inva = 1.0 / prm.a, inva2 = 1.0 / (prm.a * prm.a);
  {
    PFSH_LAUNCH("k_rhs_assemble", s);
    if (p->prec == PFSH_FP64)
      k_rhs_assemble<double><<<g, 256, 0, s>>>(p->T, B, cnt, nstride, inva, inva2, inva2, prm.nu, prm.phibar, cor, p->d_eps,
                                               (const double2 *)p->Y, (const double2 *)state, (double2 *)fE,
                                               (double2 *)fI);
    else
      k_rhs_assemble<float><<<g, 256, 0, s>>>(p->T, B, cnt, nstride, (float)inva, (float)inva2, inva2, prm.nu, prm.phibar,
                                              cor, p->d_eps32, (const float2 *)p->Y, (const double2 *)state,
                                              (double2 *)fE, (double2 *)fI);
  }
  PFSH_CHECK_LAUNCH("k_rhs_assemble");
  return PFSH_OK;
}

// ---------------------------------------------------------------------------
// implicit solve x - h L(x) = b, per coefficient (k = n(n+1)/a^2, s = 1 + h nu k)
//   zeta = b_zeta / s;  [s  h Phibar; -h k  s] [Phi; delta] = [b_Phi; b_delta]
// ---------------------------------------------------------------------------
__device__ __forceinline__ void solve3(double2 bP, double2 bz, double2 bd, double h, double k, double nu,
                                       double phibar, double2 *xP, double2 *xz, double2 *xd) {
  const double s = 1.0 + h * nu * k;
  const double det = s * s + h * h * phibar * k;
  const double id = 1.0 / det, is = 1.0 / s;
  *xP = make_double2((s * bP.x - h * phibar * bd.x) * id, (s * bP.y - h * phibar * bd.y) * id);
  *xz = make_double2(bz.x * is, bz.y * is);
  *xd = make_double2((s * bd.x + h * k * bP.x) * id, (s * bd.y + h * k * bP.y) * id);
}

__global__ void k_implicit(int T, double a, double nu, double phibar, double h, const double2 *__restrict__ b,
                           double2 *__restrict__ x) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int bb = blockIdx.y;
  const int nc = ncoef_of(T);
  if (idx >= nc) return;
  const int m = tri_m(idx, T);
  const int n = m + (idx - poff(T, m));
  const double k = (double)n * (n + 1) / (a * a);
  const double2 *in = b + (size_t)bb * 3 * nc;
  double2 *out = x + (size_t)bb * 3 * nc;
  double2 xP, xz, xd;
  solve3(in[idx], in[nc + idx], in[2 * nc + idx], h, k, nu, phibar, &xP, &xz, &xd);
  out[idx] = xP;
  out[nc + idx] = xz;
  out[2 * nc + idx] = xd;
}

int implicit_solve_launch(int T, const double *b, double *x, double h, int B, const swe_params &prm,
                          cudaStream_t s) {
  dim3 g((ncoef_of(T) + 255) / 256, B);
  {
    PFSH_LAUNCH("k_implicit", s);
    k_implicit<<<g, 256, 0, s>>>(T, prm.a, prm.nu, prm.phibar, h, (const double2 *)b, (double2 *)x);
  }
  PFSH_CHECK_LAUNCH("k_implicit");
  return PFSH_OK;
}

// ---------------------------------------------------------------------------
// SDC: constants of every node update from the old iterate, then node updates
// ---------------------------------------------------------------------------


// O_i = theta_0 + sum_j cE[i][j] FE_j + cI[i][j] FI_j (+ tau_i),  i = 1..M
// (M a template parameter: the accumulators stay in registers and no FP64
// issue slot is spent on masked-off terms).  For j = 0 and j > i both
// coefficients are dt Q[i][j] (the QE and QI corrections vanish there), so
// those terms take one FMA on S_j = FE_j + FI_j: 35 instead of 40 FP64
// operations per real component for M = 4 (the kernel is FP64-bound).
template <int M>
__global__ void __launch_bounds__(128) k_sdc_old(int nc3, int B, size_t nstride, SdcCoef c,
                                                 const double2 *__restrict__ th, const double2 *__restrict__ fe,
                                                 const double2 *__restrict__ fi, const double2 *__restrict__ tau,
                                                 size_t tstride, double2 *__restrict__ O) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nc3 * B) return;
  double2 acc[M + 1];
  const double2 t0 = th[t];
#pragma unroll
  for (int i = 1; i <= M; ++i) acc[i] = tau ? t0 + tau[(size_t)i * tstride + t] : t0;
#pragma unroll
  for (int j = 0; j <= M; ++j) {
    const double2 e = fe[(size_t)j * nstride + t], f = fi[(size_t)j * nstride + t];
    const double2 sj = make_double2(e.x + f.x, e.y + f.y);
#pragma unroll
    for (int i = 1; i <= M; ++i) {
      if (j == 0 || j > i) {
        acc[i].x = fma(c.cE[i][j], sj.x, acc[i].x);
        acc[i].y = fma(c.cE[i][j], sj.y, acc[i].y);
      } else {
        acc[i].x = fma(c.cI[i][j], f.x, fma(c.cE[i][j], e.x, acc[i].x));
        acc[i].y = fma(c.cI[i][j], f.y, fma(c.cE[i][j], e.y, acc[i].y));
      }
    }
  }
#pragma unroll
  for (int i = 1; i <= M; ++i) O[(size_t)(i - 1) * nc3 * B + t] = acc[i];
}

template <int M>
static void sdc_old_launch(int nc3, int B, size_t ns, const SdcCoef &c, const double *theta, const double *fE,
                           const double *fI, const double *tau, double *O, cudaStream_t s) {
  const size_t total = (size_t)nc3 * B;
  k_sdc_old<M><<<(unsigned)((total + 127) / 128), 128, 0, s>>>(nc3, B, ns, c, (const double2 *)theta,
                                                              (const double2 *)fE, (const double2 *)fI,
                                                              (const double2 *)tau, ns, (double2 *)O);
}

// theta_i = solve(O_i + sum_{1<=j<i} nE[i][j] FE_j^new + nI[i][j] FI_j^new, h_i)
// with the per-degree solve factors of node i precomputed in FP64:
// fac[n] = {s = 1 + h nu k, 1/s, 1/(s^2 + h^2 Phibar k), h k} for one solve;
// SPLIT (two substeps, swe_params.implicit_split): fac[n] = {1/(1 + h^2
// Phibar k), h k, h nu k, 1/s}, and with r' = r - h nu k old (old = theta_i
// of the previous iterate): x* = the nu = 0 solve of r', x = (x* + h nu k
// old) / s
template <bool SPLIT>
__global__ void __launch_bounds__(128) k_sdc_node(int T, int B, int i, size_t nstride, SdcCoef c, double hphibar,
                                                  const double4_32a *__restrict__ fac, const double2 *__restrict__ O,
                                                  const double2 *__restrict__ fe, const double2 *__restrict__ fi,
                                                  double2 *__restrict__ th) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  const int nc = ncoef_of(T);
  if (idx >= nc) return;
  const int m = tri_m(idx, T);
  const int n = m + (idx - poff(T, m));
  double2 r[3];
  for (int f = 0; f < 3; ++f) {
    const size_t t = (size_t)b * 3 * nc + f * nc + idx;
    double2 v = O[t];
    for (int j = 1; j < i; ++j) {
      const double2 e = fe[(size_t)j * nstride + t], g = fi[(size_t)j * nstride + t];
      v.x = fma(c.nI[i][j], g.x, fma(c.nE[i][j], e.x, v.x));
      v.y = fma(c.nI[i][j], g.y, fma(c.nE[i][j], e.y, v.y));
    }
    r[f] = v;
  }
  const double4_32a q = fac[n];
  double2 *out = th + (size_t)i * nstride + (size_t)b * 3 * nc;
  if (SPLIT) {
    double2 old[3];
    for (int f = 0; f < 3; ++f) {
      old[f] = out[f * nc + idx];
      r[f].x = fma(-q.z, old[f].x, r[f].x);
      r[f].y = fma(-q.z, old[f].y, r[f].y);
    }
    const double2 x0 = make_double2((r[0].x - hphibar * r[2].x) * q.x, (r[0].y - hphibar * r[2].y) * q.x);
    const double2 x2 = make_double2((r[2].x + q.y * r[0].x) * q.x, (r[2].y + q.y * r[0].y) * q.x);
    out[idx] = make_double2(fma(q.z, old[0].x, x0.x) * q.w, fma(q.z, old[0].y, x0.y) * q.w);
    out[nc + idx] = make_double2(fma(q.z, old[1].x, r[1].x) * q.w, fma(q.z, old[1].y, r[1].y) * q.w);
    out[2 * nc + idx] = make_double2(fma(q.z, old[2].x, x2.x) * q.w, fma(q.z, old[2].y, x2.y) * q.w);
    return;
  }
  out[idx] = make_double2((q.x * r[0].x - hphibar * r[2].x) * q.z, (q.x * r[0].y - hphibar * r[2].y) * q.z);
  out[nc + idx] = make_double2(r[1].x * q.y, r[1].y * q.y);
  out[2 * nc + idx] = make_double2((q.x * r[2].x + q.w * r[0].x) * q.z, (q.x * r[2].y + q.w * r[0].y) * q.z);
}

SdcCoef sdc_coef(const sdc_level *l) {
  SdcCoef c;
  const int M = l->nodes - 1;
  for (int i = 0; i < 16; ++i) {
    c.h[i] = 0.0;
    for (int j = 0; j < 16; ++j) c.cE[i][j] = c.cI[i][j] = c.nE[i][j] = c.nI[i][j] = 0.0;
  }
  const double dt = l->dt;
  for (int i = 1; i <= M; ++i) {
    for (int j = 0; j <= M; ++j) {
      const double qe = (j >= 1 && j <= i - 1) ? l->QE[i][j] : 0.0;
      const double qi = (j >= 1 && j <= i) ? l->QI[i][j] : 0.0;
      c.cE[i][j] = dt * (l->Q[i][j] - qe);
      c.cI[i][j] = dt * (l->Q[i][j] - qi);
      if (j >= 1 && j < i) {
        c.nE[i][j] = dt * l->QE[i][j];
        c.nI[i][j] = dt * l->QI[i][j];
      }
    }
    c.h[i] = dt * l->QI[i][i];
  }
  return c;
}

int sdc_sweep_strided(sdc_level *l, double *theta, double *fE, double *fI, const double *tau, size_t node_stride,
                      int B, cudaStream_t s) {
  const swe_ctx *ctx = l->ctx;
  const int T = ctx->plan->T;
  const int nc = ncoef_of(T);
  const int M = l->nodes - 1;
  if (B > l->max_batch) return fail(PFSH_EINVAL, "sdc_sweep: batch larger than the level's max_batch");
  const SdcCoef c = sdc_coef(l);
  // node stride in complex elements
  const size_t ns = node_stride / 2;
  const int nc3 = 3 * nc;
  {
    PFSH_LAUNCH("k_sdc_old", s);
    double *O = l->d_old;
    switch (M) {
      case 1: sdc_old_launch<1>(nc3, B, ns, c, theta, fE, fI, tau, O, s); break;
      case 2: sdc_old_launch<2>(nc3, B, ns, c, theta, fE, fI, tau, O, s); break;
      case 3: sdc_old_launch<3>(nc3, B, ns, c, theta, fE, fI, tau, O, s); break;
      case 4: sdc_old_launch<4>(nc3, B, ns, c, theta, fE, fI, tau, O, s); break;
      case 5: sdc_old_launch<5>(nc3, B, ns, c, theta, fE, fI, tau, O, s); break;
      case 6: sdc_old_launch<6>(nc3, B, ns, c, theta, fE, fI, tau, O, s); break;
      case 7: sdc_old_launch<7>(nc3, B, ns, c, theta, fE, fI, tau, O, s); break;
      default: sdc_old_launch<8>(nc3, B, ns, c, theta, fE, fI, tau, O, s); break;
    }
  }
  PFSH_CHECK_LAUNCH("k_sdc_old");
  for (int i = 1; i <= M; ++i) {
    dim3 g((nc + 127) / 128, B);
    if (coriolis_implicit(ctx->prm)) {
      int rc = band_sdc_node_launch(l, i, node_stride, c, l->d_old + (size_t)(i - 1) * nc3 * B * 2, fE, fI, theta, B,
                                    s);
      if (rc) return rc;
    } else {
      PFSH_LAUNCH("k_sdc_node", s);
      auto kern = ctx->prm.implicit_split ? k_sdc_node<true> : k_sdc_node<false>;
      kern<<<g, 128, 0, s>>>(T, B, i, ns, c, c.h[i] * ctx->prm.phibar,
                             (const double4_32a *)l->d_fac + (size_t)i * (T + 1),
                             (const double2 *)l->d_old + (size_t)(i - 1) * nc3 * B, (const double2 *)fE,
                             (const double2 *)fI, (double2 *)theta);
      PFSH_CHECK_LAUNCH("k_sdc_node");
    }
    int rc = rhs_eval(l->ctx, theta + (size_t)i * node_stride, fE + (size_t)i * node_stride,
                      fI + (size_t)i * node_stride, B, s);
    if (rc) return rc;
  }
  return PFSH_OK;
}

// ---------------------------------------------------------------------------
// space-time transfers between a degree-Tf and a degree-Tc triangle
// ---------------------------------------------------------------------------
struct TimeMat {
  double v[16][16];
};

// xc[i][b] = sum_k R[i][k] D(xf[k][b])   (D: keep n <= Tc)
__global__ void k_restrict(int Tf, int Tc, int B, int nf, int nc_nodes, TimeMat R, const double2 *__restrict__ xf,
                           size_t fstride, size_t fbstride, double2 *__restrict__ xc, size_t cstride) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  const int ncc = ncoef_of(Tc), ncf = ncoef_of(Tf);
  if (idx >= ncc) return;
  const int m = tri_m(idx, Tc);
  const int fidx = poff(Tf, m) + (idx - poff(Tc, m));
  {
    const int f = blockIdx.z;   // one field per grid layer
    for (int i = 0; i < nc_nodes; ++i) {
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < nf; ++k) {
        const double r = R.v[i][k];
        if (r == 0.0) continue;
        const double2 v = xf[(size_t)k * fstride + (size_t)b * fbstride + (size_t)f * ncf + fidx];
        if (r == 1.0) {
          acc = acc + v;
        } else {
          acc.x += r * v.x;
          acc.y += r * v.y;
        }
      }
      xc[(size_t)i * cstride + (size_t)b * 3 * ncc + (size_t)f * ncc + idx] = acc;
    }
  }
}

int restrict_launch(const double *Rt, int nf, int ncn, const double *xf, size_t fstride, double *xc, size_t cstride,
                    int Tf, int Tc, int B, cudaStream_t s) {
  TimeMat R;
  for (int i = 0; i < 16; ++i)
    for (int k = 0; k < 16; ++k) R.v[i][k] = (i < ncn && k < nf) ? Rt[i * 16 + k] : 0.0;
  dim3 g((ncoef_of(Tc) + 255) / 256, B, 3);
  // fbstride: batch stride inside a node (one fine state) unless broadcasting
  {
    PFSH_LAUNCH("k_restrict", s);
    k_restrict<<<g, 256, 0, s>>>(Tf, Tc, B, nf, ncn, R, (const double2 *)xf, fstride / 2,
                                 (size_t)3 * ncoef_of(Tf), (double2 *)xc, cstride / 2);
  }
  PFSH_CHECK_LAUNCH("k_restrict");
  return PFSH_OK;
}

}  // namespace pfsh
