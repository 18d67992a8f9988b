// SWE right-hand side orchestration (Sections 2-4) and IMEX-SDC levels
// (Section 5.1.1): swe_ctx_*, swe_rhs, swe_implicit_solve, sdc_level_*,
// sdc_spread, sdc_sweep.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.cuh"
#include "banded.cuh"

namespace pfsh {

// One RHS pass: velocity recovery -> synthesis of 4 fields -> inverse FFT,
// grid products, forward FFT -> analysis of 5 fields -> assembly.
// cnt, nstride: the batch is B / cnt groups of cnt consecutive states,
// nstride doubles apart (cnt = 0: contiguous; the small path needs that)
static int rhs_pass(swe_ctx *c, const double *state, double *fE, double *fI, int B, cudaStream_t s, int cnt = 0,
                    size_t nstride = 0) {
  const sht_plan *p = c->plan;
  if (small_rhs(B)) return rhs_small(p, state, fE, fI, B, c->prm, cor_args(c), s);
  int rc;
  if ((rc = rhs_prep(p, state, B, c->prm, s, cnt, nstride))) return rc;
  if ((rc = legendre_synth(p, 4 * B, s))) return rc;
  if ((rc = grid_rhs(p, B, c->prm, s))) return rc;
  if ((rc = legendre_analysis(p, 5 * B, s))) return rc;
  return rhs_assemble(p, state, fE, fI, B, c->prm, cor_args(c), s, cnt, nstride);
}

int rhs_eval(swe_ctx *c, const double *state, double *fE, double *fI, int B, cudaStream_t s) {
  const size_t st = (size_t)3 * c->plan->ncoef * 2;
  for (int b0 = 0; b0 < B; b0 += c->max_states) {
    const int nb = std::min(c->max_states, B - b0);
    int rc = rhs_pass(c, state + b0 * st, fE + b0 * st, fI ? fI + b0 * st : nullptr, nb, s);
    if (rc) return rc;
  }
  return PFSH_OK;
}

int rhs_eval_nodes(swe_ctx *c, const double *state, double *fE, double *fI, int nodes, int cnt, size_t node_stride,
                   cudaStream_t s) {
  const int B = nodes * cnt;
  if (nodes > 1 && B <= c->max_states && !small_rhs(B))
    return rhs_pass(c, state, fE, fI, B, s, cnt, node_stride);
  for (int i = 0; i < nodes; ++i) {
    const size_t o = (size_t)i * node_stride;
    int rc = rhs_eval(c, state + o, fE + o, fI ? fI + o : nullptr, cnt, s);
    if (rc) return rc;
  }
  return PFSH_OK;
}

// ---------------------------------------------------------------------------
// Gauss-Lobatto nodes and SDC matrices (host, FP64)
// ---------------------------------------------------------------------------
// Nodes on [0,1]: 0, 1 and the roots of P'_{M}(x) mapped from [-1,1], found
// by Newton iteration on P'_M with the derivative from the Legendre ODE.
static void lobatto(int nodes, double *tau) {
  const int M = nodes - 1;
  tau[0] = 0.0;
  tau[M] = 1.0;
  const double pi = 3.14159265358979323846;
  for (int i = 1; i < M; ++i) {
    double x = -std::cos(pi * i / M);  // Chebyshev-Gauss-Lobatto start
    for (int it = 0; it < 100; ++it) {
      // P_M, P_{M-1} by recurrence; P'_M and P''_M from them
      double a = 1.0, b = x;
      for (int k = 1; k < M; ++k) {
        double cc = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
        a = b;
        b = cc;
      }
      double d1 = M * (x * b - a) / (x * x - 1.0);               // P'_M
      double d2 = (2.0 * x * d1 - M * (M + 1.0) * b) / (1.0 - x * x);  // P''_M
      double dx = d1 / d2;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    tau[i] = 0.5 * (x + 1.0);
  }
}

// Lagrange basis on `src` evaluated at `dst`: out[i][j] = l_j(dst_i); entries
// within 1e-14 of 0 or 1 are snapped (nested Lobatto nodes give injection).
void lagrange_matrix(const double *src, int ns, const double *dst, int nd, double out[16][16]) {
  for (int i = 0; i < nd; ++i)
    for (int j = 0; j < ns; ++j) {
      double v = 1.0;
      for (int k = 0; k < ns; ++k)
        if (k != j) v *= (dst[i] - src[k]) / (src[j] - src[k]);
      if (std::fabs(v) < 1e-14) v = 0.0;
      if (std::fabs(v - 1.0) < 1e-14) v = 1.0;
      out[i][j] = v;
    }
}

// Q[i][j] = int_0^{tau_i} l_j: integrate the Lagrange polynomial exactly by
// expanding it in monomials.
int sdc_build_matrices(sdc_level *l, int nodes) {
  lobatto(nodes, l->tau_nodes);
  const double *t = l->tau_nodes;
  const int n = nodes;
  for (int j = 0; j < n; ++j) {
    double c[16] = {0};  // monomial coefficients of l_j
    c[0] = 1.0;
    int deg = 0;
    double den = 1.0;
    for (int k = 0; k < n; ++k) {
      if (k == j) continue;
      // multiply by (x - t_k)
      for (int d = deg + 1; d >= 1; --d) c[d] = c[d - 1] - t[k] * c[d];
      c[0] = -t[k] * c[0];
      ++deg;
      den *= (t[j] - t[k]);
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0, xp = t[i];
      for (int d = 0; d <= deg; ++d) {
        s += c[d] * xp / (d + 1);
        xp *= t[i];
      }
      l->Q[i][j] = s / den;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) l->QE[i][j] = (j < i) ? t[j + 1] - t[j] : 0.0;
  // QI = [[0,0],[0,U^T]] with Q[1:,1:]^T = L U (Doolittle, no pivoting)
  const int m = n - 1;
  double A[16][16], L[16][16], U[16][16];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      A[i][j] = l->Q[j + 1][i + 1];
      L[i][j] = (i == j) ? 1.0 : 0.0;
      U[i][j] = 0.0;
    }
  for (int i = 0; i < m; ++i) {
    for (int k = i; k < m; ++k) {
      double s = A[i][k];
      for (int q = 0; q < i; ++q) s -= L[i][q] * U[q][k];
      U[i][k] = s;
    }
    if (U[i][i] == 0.0) return fail(PFSH_EINVAL, "sdc: LU of Q^T needs pivoting");
    for (int k = i + 1; k < m; ++k) {
      double s = A[k][i];
      for (int q = 0; q < i; ++q) s -= L[k][q] * U[q][i];
      L[k][i] = s / U[i][i];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) l->QI[i][j] = (i >= 1 && j >= 1) ? U[j - 1][i - 1] : 0.0;
  return PFSH_OK;
}

}  // namespace pfsh

using namespace pfsh;

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" int swe_ctx_create(swe_ctx **out, sht_plan *plan, const swe_params *prm) {
  if (!out || !plan || !prm) return fail(PFSH_EINVAL, "swe_ctx_create: NULL argument");
  if (!(prm->a > 0) || !(prm->nu >= 0)) return fail(PFSH_EINVAL, "swe_ctx_create: need a > 0, nu >= 0");
  if (prm->coriolis != PFSH_CORIOLIS_EXPLICIT && prm->coriolis != PFSH_CORIOLIS_IMPLICIT)
    return fail(PFSH_EINVAL, "swe_ctx_create: coriolis must be PFSH_CORIOLIS_EXPLICIT or PFSH_CORIOLIS_IMPLICIT");
  if (prm->implicit_split != 0 && prm->implicit_split != 1)
    return fail(PFSH_EINVAL, "swe_ctx_create: implicit_split must be 0 or 1");
  if (plan->max_batch < 5) return fail(PFSH_EINVAL, "swe_ctx_create: plan max_batch must be >= 5");
  if (plan->prec == PFSH_FP16)
    return fail(PFSH_EUNSUPPORTED, "swe_ctx_create: the FP16 form serves transforms only (the flux products "
                                   "of the right-hand side exceed the fp16 range)");
  swe_ctx *c = new (std::nothrow) swe_ctx();
  if (!c) return fail(PFSH_ENOMEM, "swe_ctx_create");
  c->plan = plan;
  c->prm = *prm;
  c->max_states = plan->max_batch / 5;
  if (coriolis_implicit(c->prm)) {
    int rc = band_ctx_init(c);
    if (rc) { delete c; return rc; }
  }
  *out = c;
  return PFSH_OK;
}

extern "C" int swe_ctx_destroy(swe_ctx *c) {
  delete c;
  return PFSH_OK;
}

extern "C" int swe_rhs(swe_ctx *c, const double *state, double *fE, double *fI, int B, pfsh_stream_t stream) {
  if (!c || B < 0 || (B > 0 && (!state || !fE))) return fail(PFSH_EINVAL, "swe_rhs: invalid argument");
  if (B == 0) return PFSH_OK;
  const size_t n = (size_t)B * 3 * c->plan->ncoef * 2;
  int rc = rhs_eval(c, state, fE, fI, B, (cudaStream_t)stream);
  if (!rc) rc = check_finite(fE, n, (cudaStream_t)stream);
  if (!rc && fI) rc = check_finite(fI, n, (cudaStream_t)stream);
  return rc;
}

extern "C" int swe_implicit_solve(swe_ctx *c, const double *b, double *x, double h, int B, pfsh_stream_t stream) {
  if (!c || B < 0 || (B > 0 && (!b || !x)) || !(h >= 0)) return fail(PFSH_EINVAL, "swe_implicit_solve: invalid argument");
  if (B == 0) return PFSH_OK;
  if (coriolis_implicit(c->prm)) return band_solve_launch(c, b, x, h, B, (cudaStream_t)stream);
  return implicit_solve_launch(c->plan->T, b, x, h, B, c->prm, (cudaStream_t)stream);
}

extern "C" int sdc_level_create(sdc_level **out, swe_ctx *ctx, int nodes, double dt, int max_batch) {
  if (!out || !ctx) return fail(PFSH_EINVAL, "sdc_level_create: NULL argument");
  *out = nullptr;
  if (nodes < 2 || nodes > 9) return fail(PFSH_EINVAL, "sdc_level_create: nodes must be in 2..9");
  if (!(dt > 0) || max_batch < 1) return fail(PFSH_EINVAL, "sdc_level_create: need dt > 0, max_batch >= 1");
  sdc_level *l = new (std::nothrow) sdc_level();
  if (!l) return fail(PFSH_ENOMEM, "sdc_level_create");
  l->ctx = ctx;
  l->nodes = nodes;
  l->dt = dt;
  l->max_batch = max_batch;
  int rc = sdc_build_matrices(l, nodes);
  if (rc) { delete l; return rc; }
  size_t bytes = (size_t)(nodes - 1) * max_batch * 3 * ctx->plan->ncoef * 16;
  const int T = ctx->plan->T;
  if (cudaMalloc(&l->d_old, bytes) != cudaSuccess || cudaMalloc(&l->d_fac, (size_t)nodes * (T + 1) * 32) != cudaSuccess) {
    cudaGetLastError();
    if (l->d_old) cudaFree(l->d_old);
    delete l;
    return fail(PFSH_ENOMEM, "sdc_level_create: workspace");
  }
  {
    // implicit solve of node i (h = dt QI[i][i]) per degree n, k = n(n+1)/a^2:
    // one solve:  s = 1 + h nu k, 1/s, 1/(s^2 + h^2 Phibar k), h k
    // two substeps (swe_params.implicit_split): 1/(1 + h^2 Phibar k), h k,
    //             h nu k, 1/s
    std::vector<double> fac((size_t)nodes * (T + 1) * 4, 0.0);
    const swe_params &pr = ctx->prm;
    for (int i = 0; i < nodes; ++i) {
      const double h = dt * l->QI[i][i];
      for (int n = 0; n <= T; ++n) {
        const double k = (double)n * (n + 1) / (pr.a * pr.a);
        const double sv = 1.0 + h * pr.nu * k;
        double *f = &fac[((size_t)i * (T + 1) + n) * 4];
        if (pr.implicit_split) {
          f[0] = 1.0 / (1.0 + h * h * pr.phibar * k);
          f[1] = h * k;
          f[2] = h * pr.nu * k;
          f[3] = 1.0 / sv;
        } else {
          f[0] = sv;
          f[1] = 1.0 / sv;
          f[2] = 1.0 / (sv * sv + h * h * pr.phibar * k);
          f[3] = h * k;
        }
      }
    }
    if (cudaMemcpy(l->d_fac, fac.data(), fac.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(l->d_old);
      cudaFree(l->d_fac);
      delete l;
      return fail(PFSH_ECUDA, "sdc_level_create: factors");
    }
  }
  if (coriolis_implicit(ctx->prm)) {
    // banded-solve factors of nodes 1..M (h = dt QI[i][i]), computed on the device
    const size_t per = band_table_entries(ctx->plan->ncoef);
    int rc2 = PFSH_OK;
    if (cudaMalloc(&l->d_band, (size_t)nodes * per * sizeof(double4_32a)) != cudaSuccess) {
      cudaGetLastError();
      rc2 = fail(PFSH_ENOMEM, "sdc_level_create: banded factors");
    }
    for (int i = 1; i < nodes && rc2 == PFSH_OK; ++i)
      rc2 = band_factor_launch(ctx, dt * l->QI[i][i], ctx->prm.implicit_split ? 0.0 : ctx->prm.nu,
                               l->d_band + (size_t)i * per, 0);
    if (rc2 == PFSH_OK && cudaDeviceSynchronize() != cudaSuccess) rc2 = fail(PFSH_ECUDA, "sdc_level_create: factors");
    if (rc2) {
      cudaFree(l->d_old);
      cudaFree(l->d_fac);
      if (l->d_band) cudaFree(l->d_band);
      delete l;
      return rc2;
    }
  }
  *out = l;
  return PFSH_OK;
}

extern "C" int sdc_level_destroy(sdc_level *l) {
  if (!l) return PFSH_OK;
  cudaDeviceSynchronize();
  if (l->d_old) cudaFree(l->d_old);
  if (l->d_fac) cudaFree(l->d_fac);
  if (l->d_band) cudaFree(l->d_band);
  delete l;
  return PFSH_OK;
}

extern "C" int sdc_spread(sdc_level *l, const double *theta0, double *theta, double *fE, double *fI, int B,
                          pfsh_stream_t stream) {
  if (!l || B < 0 || (B > 0 && (!theta0 || !theta || !fE || !fI))) return fail(PFSH_EINVAL, "sdc_spread: invalid argument");
  if (B == 0) return PFSH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t st = (size_t)3 * l->ctx->plan->ncoef * 2 * B;  // doubles per node
  PFSH_CUDA(cudaMemcpyAsync(theta, theta0, st * 8, cudaMemcpyDeviceToDevice, s));
  int rc = rhs_eval(l->ctx, theta, fE, fI, B, s);
  if (rc) return rc;
  for (int i = 1; i < l->nodes; ++i) {
    PFSH_CUDA(cudaMemcpyAsync(theta + i * st, theta0, st * 8, cudaMemcpyDeviceToDevice, s));
    PFSH_CUDA(cudaMemcpyAsync(fE + i * st, fE, st * 8, cudaMemcpyDeviceToDevice, s));
    PFSH_CUDA(cudaMemcpyAsync(fI + i * st, fI, st * 8, cudaMemcpyDeviceToDevice, s));
  }
  return PFSH_OK;
}

extern "C" int sdc_sweep(sdc_level *l, double *theta, double *fE, double *fI, const double *tau, int B,
                         pfsh_stream_t stream) {
  if (!l || B < 0 || (B > 0 && (!theta || !fE || !fI))) return fail(PFSH_EINVAL, "sdc_sweep: invalid argument");
  if (B == 0) return PFSH_OK;
  const size_t st = (size_t)3 * l->ctx->plan->ncoef * 2 * B;
  int rc = sdc_sweep_strided(l, theta, fE, fI, tau, st, B, (cudaStream_t)stream);
  if (!rc) rc = check_finite(theta, st * l->nodes, (cudaStream_t)stream);
  return rc;
}
