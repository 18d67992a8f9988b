// The split with the Coriolis term implicit (F_I = L + C, F_E = N evaluated
// with eta = zeta; Section 4 keeps the Coriolis term explicit, in N).
//
// Linear Coriolis tendency C = [0, -div(f V), curl(f V)], f = 2 Omega mu.
// With V = k x grad psi + grad chi, -div(f V) = -f delta - 2 Omega V/a and
// curl(f V) = f zeta - 2 Omega U/a (U = u cos(phi), V = v cos(phi)), where
// only the Laplacians of psi and chi enter (no n = 0 coefficient).  The
// multiplication by mu couples degree n to n +- 1 within an order m:
//   C_zeta,n  = 2 Omega [ i m/(n(n+1)) zeta_n - alpha_n delta_{n-1} - beta_n delta_{n+1} ]
//   C_delta,n = 2 Omega [ i m/(n(n+1)) delta_n + alpha_n zeta_{n-1} + beta_n zeta_{n+1} ]
//   alpha_n = eps_n (n+1)/n for n >= 2 (0 for n <= 1),  beta_n = eps_{n+1} n/(n+1) (0 at n = T).
//
// Implicit system x - h (L + C)(x) = b of one order m (Eq. implicit_systems
// with the Coriolis coupling): with k_n = n(n+1)/a^2, s_n = 1 + h nu k_n and
// th = 2 Omega h, eliminating Phi_n = (b_Phi,n - h Phibar delta_n) / s_n gives
//   zeta row:  (s_n - i th m/(n(n+1))) zeta_n + th alpha_n delta_{n-1} + th beta_n delta_{n+1} = b_zeta,n
//   delta row: (d_n - i th m/(n(n+1))) delta_n - th alpha_n zeta_{n-1} - th beta_n zeta_{n+1}
//              = b_delta,n + (h k_n / s_n) b_Phi,n,            d_n = s_n + h^2 Phibar k_n / s_n,
// two independent tridiagonal chains, (zeta_m, delta_{m+1}, zeta_{m+2}, ...)
// and (delta_m, zeta_{m+1}, ...).  Scaled by the kinetic-energy weights
// 1/(n(n+1)) the Coriolis coupling is skew-Hermitian and the diagonal has a
// positive real part, so elimination without pivoting is stable for any h.
// Chain c, position j: degree n = m + j, field (j + c) & 1 (0 zeta, 1 delta).
// Forward elimination with w_j = D_j - a_j c'_{j-1}, c'_j = c_j / w_j,
// y_j = (r_j - a_j y_{j-1}) / w_j, then x_j = y_j - c'_j x_{j+1}.
// The factors {c'_j, 1/w_j} and the forward coefficients al_j = -a_j / w_j
// depend on h only: one table per SDC node (band_table_entries); the two
// substitution passes run as warp scans (band_chain_scan).
#pragma once

#include "internal.cuh"

namespace pfsh {

// eps_n^m = sqrt((n^2 - m^2) / (4 n^2 - 1)) (0 for n = 0 or n < m); the
// context's coupling table CorArgs::ab holds {alpha_n, beta_n, m/(n(n+1)), 0}
// per packed coefficient (band_ctx_init)
__host__ __device__ inline double band_eps(int n, int m) {
  return (n > 0 && n >= m) ? sqrt((double)(n - m) * (double)(n + m) / (4.0 * n * n - 1.0)) : 0.0;
}

// C of coefficient (m, n) (packed index idx) of one state [3][nc]
__device__ __forceinline__ void coriolis_point(int m, int n, int T, const double2 *__restrict__ st, int nc,
                                               size_t idx, CorArgs cor, double2 *cz, double2 *cd) {
  const double4_32a q = cor.ab[idx];
  auto at = [&](int f, int nn, int off) {
    if (nn < m || nn > T) return make_double2(0.0, 0.0);
    double2 v = st[(size_t)f * nc + idx + off];
    if (m == 0) v.y = 0.0;
    return v;
  };
  const double2 z = at(1, n, 0), d = at(2, n, 0);
  const double2 zm = at(1, n - 1, -1), dm = at(2, n - 1, -1), zp = at(1, n + 1, 1), dp = at(2, n + 1, 1);
  const double tw = cor.tw;
  *cz = make_double2(tw * (-q.z * z.y - q.x * dm.x - q.y * dp.x), tw * (q.z * z.x - q.x * dm.y - q.y * dp.y));
  *cd = make_double2(tw * (-q.z * d.y + q.x * zm.x + q.y * zp.x), tw * (q.z * d.x + q.x * zm.y + q.y * zp.y));
}

// factor table of one step size, in double4 units: [2][nc] {c', 1/w} (rows
// of zeta, then of delta) followed by [2][nc] complex al = -a/w, packed two
// per double4
__host__ __device__ inline size_t band_table_entries(int nc) { return (size_t)3 * nc; }

// shared-memory scratch of one order's banded solve besides its right-hand
// sides (K = T+1 at most): factors [2][K], forward coefficients [2][K], plus
// alignment slack
__host__ __device__ inline size_t band_scratch_bytes(int T) {
  return (size_t)(T + 1) * (2 * sizeof(double4_32a) + 2 * sizeof(double2)) + 32;
}

// complex FP64 helpers of the chain scans
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 zfma(double2 a, double2 b, double2 c) {   // a b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 zshfl_up(double2 v, int d) {
  return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 zshfl_down(double2 v, int d) {
  return make_double2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// One chain (c) of an order, solved by one warp.  Both elimination passes
// are first-order affine recurrences,
//   forward  y_j = al_j y_{j-1} + be_j,  al_j = -a_j / w_j, be_j = r_j / w_j,  y_{-1} = 0
//   backward x_j = ga_j x_{j+1} + y_j,   ga_j = -c'_j,                        x_K = 0,
// evaluated as scans: lane l takes the segment [l S, (l+1) S) (S = ceil(K/32)),
// composes its affine maps, the lanes combine the composites in log2(32)
// shuffle steps, and each lane re-runs its segment from its incoming value.
// A sequential elimination would chain K dependent FP64 steps; this chains
// about 2 S + 5.  sr[1 + field][j] holds r on entry, x on return (be_j in
// between); stab [2][K] {c', 1/w}, sal [2][K] al, by field.
__device__ __forceinline__ void band_chain_scan(int c, int lane, int K, const double4_32a *stab, const double2 *sal,
                                                double2 *sr) {
  const int S = (K + 31) >> 5, j0 = min(K, lane * S), j1 = min(K, j0 + S);
  // forward: composite of the lane's maps, inclusive scan, re-run
  double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);
  for (int j = j0; j < j1; ++j) {
    const int f = (j + c) & 1;
    const double4_32a q = stab[f * K + j];
    double2 *p = sr + (1 + f) * K + j;
    const double2 al = sal[f * K + j], be = zmul(*p, make_double2(q.z, q.w));
    *p = be;
    A = zmul(al, A);
    B = zfma(al, B, be);
  }
  for (int d = 1; d < 32; d <<= 1) {
    const double2 Ap = zshfl_up(A, d), Bp = zshfl_up(B, d);
    if (lane >= d) {
      B = zfma(A, Bp, B);
      A = zmul(A, Ap);
    }
  }
  double2 y = zshfl_up(B, 1);
  if (lane == 0) y = make_double2(0.0, 0.0);
  for (int j = j0; j < j1; ++j) {
    const int f = (j + c) & 1;
    double2 *p = sr + (1 + f) * K + j;
    y = zfma(sal[f * K + j], y, *p);
    *p = y;
  }
  // backward: maps x_{j+1} -> x_j composed from the right, suffix scan, re-run
  A = make_double2(1.0, 0.0);
  B = make_double2(0.0, 0.0);
  for (int j = j1 - 1; j >= j0; --j) {
    const int f = (j + c) & 1;
    const double4_32a q = stab[f * K + j];
    const double2 ga = make_double2(-q.x, -q.y);
    A = zmul(ga, A);
    B = zfma(ga, B, sr[(1 + f) * K + j]);
  }
  for (int d = 1; d < 32; d <<= 1) {
    const double2 An = zshfl_down(A, d), Bn = zshfl_down(B, d);
    if (lane + d < 32) {
      B = zfma(A, Bn, B);
      A = zmul(A, An);
    }
  }
  double2 x = zshfl_down(B, 1);
  if (lane == 31) x = make_double2(0.0, 0.0);
  for (int j = j1 - 1; j >= j0; --j) {
    const int f = (j + c) & 1;
    const double4_32a q = stab[f * K + j];
    double2 *p = sr + (1 + f) * K + j;
    x = zfma(make_double2(-q.x, -q.y), x, *p);
    *p = x;
  }
}

// Solve the order-m system in place.  sr[3][K] (Phi, zeta, delta rows of
// order m, K = T+1-m) holds b on entry and x on return; tab = the factor table
// of the step size (band_table_entries); scratch = band_scratch_bytes(T) of
// shared memory (any 16-byte alignment).  The per-degree constants of the Phi
// elimination, g = h k / s and 1/s, come from the SDC node's factors `fac`
// (layouts of k_sdc_node: one solve {s, 1/s, 1/det, h k}; `fac_split`
// {1/det0, h k, h nu k, 1/s}, whose banded solve has nu = 0) or, with fac =
// nullptr, are computed from h and nu.  Called by every thread of a block of
// at least 64 threads (warps 0 and 1 solve the two chains); ends with a
// barrier.
__device__ __forceinline__ void band_order_solve(int m, int T, double h, double inva2, double nu, double phibar,
                                                 CorArgs cor, const double4_32a *__restrict__ tab,
                                                 const double4_32a *__restrict__ fac, bool fac_split, double2 *sr,
                                                 void *scratch) {
  const int K = T + 1 - m, p0 = poff(T, m), nc = ncoef_of(T);
  double4_32a *stab = reinterpret_cast<double4_32a *>((reinterpret_cast<uintptr_t>(scratch) + 31) & ~uintptr_t(31));
  double2 *sal = reinterpret_cast<double2 *>(stab + 2 * K);   // [2][K]
  const double2 *tal = reinterpret_cast<const double2 *>(tab + 2 * (size_t)nc);
  auto consts = [&](int n, double *g, double *is) {
    if (fac) {
      const double4_32a q = fac[n];
      *g = fac_split ? q.y : q.w * q.y;
      *is = fac_split ? 1.0 : q.y;
    } else {
      const double k = (double)n * (n + 1) * inva2;
      *is = 1.0 / (1.0 + h * nu * k);
      *g = h * k * *is;
    }
  };
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    double g, is;
    consts(m + j, &g, &is);
    const double2 bP = sr[j];
    sr[2 * K + j].x = fma(g, bP.x, sr[2 * K + j].x);
    sr[2 * K + j].y = fma(g, bP.y, sr[2 * K + j].y);
    stab[j] = tab[p0 + j];
    stab[K + j] = tab[(size_t)nc + p0 + j];
    sal[j] = tal[p0 + j];
    sal[K + j] = tal[(size_t)nc + p0 + j];
  }
  __syncthreads();
  if (threadIdx.x < 64) band_chain_scan(threadIdx.x >> 5, threadIdx.x & 31, K, stab, sal, sr);
  __syncthreads();
  const double hp = h * phibar;
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    double g, is;
    consts(m + j, &g, &is);
    const double2 bP = sr[j], d = sr[2 * K + j];
    sr[j] = make_double2((bP.x - hp * d.x) * is, (bP.y - hp * d.y) * is);
  }
  __syncthreads();
}

}  // namespace pfsh
