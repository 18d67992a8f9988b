// Banded implicit solve of the split with the Coriolis term implicit (the
// operator and the elimination are described in banded.cuh): the context's
// coupling table, the factor tables of one step size h, and the per-order
// solve for swe_implicit_solve and for the node updates of an SDC sweep.
#include <vector>

#include "internal.cuh"
#include "banded.cuh"

namespace pfsh {

// Factors {c'_j, 1/w_j} and forward coefficients al_j = -a_j / w_j of both
// chains of every order for step size h: thread (m, c) runs the elimination
// of chain c of order m.  tab: band_table_entries(nc) (see banded.cuh).
__global__ void k_band_factor(int T, double h, double inva2, double nu, double phibar, CorArgs cor,
                              double4_32a *__restrict__ tab) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * (T + 1)) return;
  const int m = t >> 1, c = t & 1, K = T + 1 - m, p0 = poff(T, m), nc = ncoef_of(T);
  double2 *tal = reinterpret_cast<double2 *>(tab + 2 * (size_t)nc);
  const double th = cor.tw * h;
  double2 cp = make_double2(0.0, 0.0);
  for (int j = 0; j < K; ++j) {
    const int n = m + j, f = (j + c) & 1;
    const double k = (double)n * (n + 1) * inva2, s = 1.0 + h * nu * k;
    const double4_32a q = cor.ab[p0 + j];
    const double sg = f ? -th : th, a = sg * q.x, cc = sg * q.y;
    const double wx = (f ? s + h * h * phibar * k / s : s) - a * cp.x, wy = -th * q.z - a * cp.y;
    const double r = 1.0 / (wx * wx + wy * wy);
    const double iwx = wx * r, iwy = -wy * r;
    cp = make_double2(cc * iwx, cc * iwy);
    double4_32a o;
    o.x = cp.x;
    o.y = cp.y;
    o.z = iwx;
    o.w = iwy;
    const size_t e = (size_t)f * nc + p0 + j;
    tab[e] = o;
    tal[e] = make_double2(-a * iwx, -a * iwy);
  }
}

// right-hand sides [3][T+1] of one order, rounded up to 32 bytes
__host__ __device__ inline size_t band_rhs_bytes(int T) {
  return ((size_t)3 * (T + 1) * sizeof(double2) + 31) & ~size_t(31);
}

// One block per (order m, state b).  SDC = false: x = solve(b) (in may alias
// out: the block reads its whole column before writing).  SDC = true: the
// right-hand side of node i is O_i + sum_{1<=j<i} nE[i][j] F_E,j + nI[i][j]
// F_I,j (in = O of node i [B][3nc], fe/fi node-major with stride ns) and the
// result goes to out = theta of node i; fac = the node's solve factors
// (k_sdc_node layouts).  SPLIT (with SDC): two substeps, x* = the nu = 0 solve
// of r - h nu k old (tab built with nu = 0), then x = (x* + h nu k old) / s,
// old = theta of node i on entry.
template <bool SDC, bool SPLIT>
__global__ void __launch_bounds__(128) k_band_node(int T, int i, size_t ns, SdcCoef coef, double h, double inva2,
                                                   double nu, double phibar, CorArgs cor,
                                                   const double4_32a *__restrict__ tab,
                                                   const double4_32a *__restrict__ fac, const double2 *in,
                                                   const double2 *__restrict__ fe, const double2 *__restrict__ fi,
                                                   double2 *out) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  const int m = blockIdx.x, b = blockIdx.y, K = T + 1 - m, nc = ncoef_of(T), p0 = poff(T, m);
  double2 *sr = reinterpret_cast<double2 *>(smem_raw);
  const size_t base = (size_t)b * 3 * nc + p0;
  for (int t = threadIdx.x; t < 3 * K; t += blockDim.x) {
    const int f = t / K;
    const size_t e = base + (size_t)f * nc + (t - f * K);
    double2 v = in[e];
    if (SDC) {
      for (int j = 1; j < i; ++j) {
        const double2 a = fe[(size_t)j * ns + e], g = fi[(size_t)j * ns + e];
        v.x = fma(coef.nI[i][j], g.x, fma(coef.nE[i][j], a.x, v.x));
        v.y = fma(coef.nI[i][j], g.y, fma(coef.nE[i][j], a.y, v.y));
      }
    }
    if (SPLIT) {   // r - h nu k old
      const double hnk = fac[m + (t - f * K)].z;
      const double2 o = out[e];
      v.x = fma(-hnk, o.x, v.x);
      v.y = fma(-hnk, o.y, v.y);
    }
    sr[t] = v;
  }
  __syncthreads();
  band_order_solve(m, T, h, inva2, SPLIT ? 0.0 : nu, phibar, cor, tab, fac, SPLIT, sr,
                   smem_raw + band_rhs_bytes(T));
  for (int t = threadIdx.x; t < 3 * K; t += blockDim.x) {
    const int f = t / K;
    const size_t e = base + (size_t)f * nc + (t - f * K);
    double2 x = sr[t];
    if (SPLIT) {   // (x* + h nu k old) / s
      const double4_32a q = fac[m + (t - f * K)];
      const double2 o = out[e];
      x = make_double2(fma(q.z, o.x, x.x) * q.w, fma(q.z, o.y, x.y) * q.w);
    }
    out[e] = x;
  }
}

int band_ctx_init(swe_ctx *c) {
  const int T = c->plan->T, nc = c->plan->ncoef;
  std::vector<double> ab((size_t)nc * 4, 0.0);
  for (int m = 0; m <= T; ++m)
    for (int n = m; n <= T; ++n) {
      double *q = &ab[((size_t)poff(T, m) + (n - m)) * 4];
      q[0] = n >= 2 ? band_eps(n, m) * (n + 1) / n : 0.0;
      q[1] = n < T ? band_eps(n + 1, m) * n / (n + 1) : 0.0;
      q[2] = n > 0 ? (double)m / ((double)n * (n + 1)) : 0.0;
    }
  if (cudaMalloc(&c->d_cor, (size_t)nc * sizeof(double4_32a)) != cudaSuccess ||
      cudaMalloc(&c->d_band_scr, band_table_entries(nc) * sizeof(double4_32a)) != cudaSuccess) {
    cudaGetLastError();
    return fail(PFSH_ENOMEM, "swe_ctx_create: Coriolis tables");
  }
  if (cudaMemcpy(c->d_cor, ab.data(), ab.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return fail(PFSH_ECUDA, "swe_ctx_create: Coriolis tables");
  }
  return PFSH_OK;
}

int band_factor_launch(const swe_ctx *c, double h, double nu, double4_32a *tab, cudaStream_t s) {
  const int T = c->plan->T;
  const swe_params &p = c->prm;
  {
    PFSH_LAUNCH("k_band_factor", s);
    k_band_factor<<<(2 * (T + 1) + 63) / 64, 64, 0, s>>>(T, h, 1.0 / (p.a * p.a), nu, p.phibar, cor_args(c), tab);
  }
  PFSH_CHECK_LAUNCH("k_band_factor");
  return PFSH_OK;
}

template <bool SDC, bool SPLIT>
static int band_node_launch(const swe_ctx *c, int i, size_t ns, const SdcCoef &coef, double h,
                            const double4_32a *tab, const double4_32a *fac, const double *in, const double *fe,
                            const double *fi, double *out, int B, cudaStream_t s) {
  const int T = c->plan->T;
  const swe_params &p = c->prm;
  const size_t smem = band_rhs_bytes(T) + band_scratch_bytes(T);
  int rc = ensure_smem((const void *)k_band_node<SDC, SPLIT>, smem);
  if (rc) return rc;
  {
    PFSH_LAUNCH("k_band_node", s);
    k_band_node<SDC, SPLIT><<<dim3(T + 1, B), 128, smem, s>>>(T, i, ns, coef, h, 1.0 / (p.a * p.a), p.nu, p.phibar,
                                                       cor_args(c), tab, fac, (const double2 *)in, (const double2 *)fe,
                                                       (const double2 *)fi, (double2 *)out);
  }
  PFSH_CHECK_LAUNCH("k_band_node");
  return PFSH_OK;
}

int band_solve_launch(const swe_ctx *c, const double *b, double *x, double h, int B, cudaStream_t s) {
  int rc = band_factor_launch(c, h, c->prm.nu, c->d_band_scr, s);
  if (rc) return rc;
  SdcCoef none = {};
  return band_node_launch<false, false>(c, 0, 0, none, h, c->d_band_scr, nullptr, b, nullptr, nullptr, x, B, s);
}

int band_sdc_node_launch(const sdc_level *l, int i, size_t node_stride, const SdcCoef &coef, const double *O,
                         const double *fE, const double *fI, double *theta, int B, cudaStream_t s) {
  const swe_ctx *c = l->ctx;
  auto launch = c->prm.implicit_split ? band_node_launch<true, true> : band_node_launch<true, false>;
  return launch(c, i, node_stride / 2, coef, coef.h[i], l->d_band + (size_t)i * band_table_entries(c->plan->ncoef),
                (const double4_32a *)l->d_fac + (size_t)i * (c->plan->T + 1), O, fE, fI,
                theta + (size_t)i * node_stride, B, s);
}

}  // namespace pfsh

swe_ctx::~swe_ctx() {
  if (d_cor || d_band_scr) cudaDeviceSynchronize();
  if (d_cor) cudaFree(d_cor);
  if (d_band_scr) cudaFree(d_band_scr);
}
