// Per-coefficient spectral operations shared by the batched and the
// small-batch RHS kernels (Section 2):
//
//   prep:     eta = zeta + 2 Omega mu, Phi' = Phi - Phibar, and U = u cos(phi),
//             V = v cos(phi) from psi = -a^2 zeta/(n(n+1)), chi likewise:
//             U_n = [(n-1) eps_n psi_{n-1} - (n+2) eps_{n+1} psi_{n+1} + i m chi_n] / a
//             V_n = [i m psi_n - (n-1) eps_n chi_{n-1} + (n+2) eps_{n+1} chi_{n+1}] / a
//   assemble: div_n  = [i m A_n + n eps_{n+1} B_{n+1} - (n+1) eps_n B_{n-1}] / a
//             curl_n = [i m B_n - n eps_{n+1} A_{n+1} + (n+1) eps_n A_{n-1}] / a
//             F_E = [-div(A2,B2), -div(A1,B1), curl(A1,B1) + n(n+1)/a^2 E]
//             F_I = [-Phibar delta - nu k Phi, -nu k zeta, k Phi - nu k delta]
//             (+ the Coriolis tendency C when it is implicit, banded.cuh)
//
// The arithmetic type M is the plan's transform type: double for FP64 plans;
// float for the mixed plans, whose transforms consume and produce float data
// anyway (FP64 is a scarce pipe on this GPU).  The mean subtraction of the
// (0,0) geopotential coefficient and F_I are always computed in double.
#pragma once

#include "internal.cuh"
#include "banded.cuh"

namespace pfsh {

template <typename M> struct SpecTables {
  const M *eps;    // [ext row] eps_n^m of the extended triangle
  const M *ilap;   // [n] 1/(n(n+1)), 0 at n = 0
};

template <typename M>
__device__ __forceinline__ typename cpx<M>::t ld(const double2 *p) {
  const double2 v = *p;
  typename cpx<M>::t r;
  r.x = from_double<M>(v.x);
  r.y = from_double<M>(v.y);
  return r;
}

// X values (eta, Phi', U, V) of coefficient (m, n), n <= T+1, of one state.
// `base` = packed index of (m, 0) minus... i.e. packed(m, n') = base + n';
// `erow` = extended-triangle row of (m, n).
template <typename M>
__device__ __forceinline__ void prep_point(int T, int m, int n, const double2 *__restrict__ Phi,
                                           const double2 *__restrict__ zeta, const double2 *__restrict__ delta,
                                           int base, size_t erow, SpecTables<M> tb, M ma2, M inva, double omega,
                                           double phibar, typename cpx<M>::t out[4]) {
  typedef typename cpx<M>::t C;
  auto pc = [&](int nn, C *ps, C *ch) {
    if (nn < m || nn > T || nn == 0) {
      *ps = mk<C>(0.0, 0.0);
      *ch = mk<C>(0.0, 0.0);
      return;
    }
    const M f = ma2 * tb.ilap[nn];
    C z = ld<M>(zeta + base + nn), d = ld<M>(delta + base + nn);
    if (m == 0) { z.y = 0; d.y = 0; }
    ps->x = f * z.x; ps->y = f * z.y;
    ch->x = f * d.x; ch->y = f * d.y;
  };
  C eta = mk<C>(0.0, 0.0), php = mk<C>(0.0, 0.0);
  if (n <= T) {
    if (m == 0 && n <= 1) {
      double2 e = zeta[base + n], q = Phi[base + n];
      if (n == 1) e.x += 2.0 * omega * 0.81649658092772603273;   // 2 Omega mu, mu = P_1^0 / sqrt(3/2)
      if (n == 0) q.x -= 1.41421356237309504880 * phibar;        // 1 = sqrt(2) P_0^0
      eta.x = from_double<M>(e.x);
      eta.y = 0;
      php.x = from_double<M>(q.x);
      php.y = 0;
    } else {
      eta = ld<M>(zeta + base + n);
      php = ld<M>(Phi + base + n);
      if (m == 0) { eta.y = 0; php.y = 0; }
    }
  }
  C psm, chm, ps0, ch0, psp, chp;
  pc(n - 1, &psm, &chm);
  pc(n, &ps0, &ch0);
  pc(n + 1, &psp, &chp);
  const M cm = (M)(n - 1) * tb.eps[erow];
  const M cp = (n <= T) ? (M)(n + 2) * tb.eps[erow + 1] : (M)0;
  const M mm = (M)m;
  out[0] = eta;
  out[1] = php;
  out[2] = mk<C>((cm * psm.x - cp * psp.x - mm * ch0.y) * inva, (cm * psm.y - cp * psp.y + mm * ch0.x) * inva);
  out[3] = mk<C>((-mm * ps0.y - cm * chm.x + cp * chp.x) * inva, (mm * ps0.x - cm * chm.y + cp * chp.y) * inva);
}

// F_E of coefficient (m, n <= T) from analysed rows: y(i, f) returns the
// analysed value of field f (A1, B1, A2, B2, E) at degree n - m + i - 1... see
// callers: cur/up/dn give rows n, n+1, n-1 (dn valid only if n > m).
template <typename M, typename C>
__device__ __forceinline__ void assemble_point(int m, int n, const C cur[5], const C up[5], const C dn[5], bool has_dn,
                                               M eps_up, M eps_n, M inva, M inva2, double2 fe[3]) {
  const M cu = (M)n * eps_up, cd = (M)(n + 1) * eps_n;
  const M mm = (M)m;
  const C z = mk<C>(0.0, 0.0);
  const C A1 = cur[0], B1 = cur[1], A2 = cur[2], E = cur[4];
  const C A1u = up[0], B1u = up[1], B2u = up[3];
  const C A1d = has_dn ? dn[0] : z, B1d = has_dn ? dn[1] : z, B2d = has_dn ? dn[3] : z;
  const M k = (M)n * (M)(n + 1) * inva2;
  fe[0] = make_double2(to_double<M>(-(-mm * A2.y + cu * B2u.x - cd * B2d.x) * inva),
                       to_double<M>(-(mm * A2.x + cu * B2u.y - cd * B2d.y) * inva));
  fe[1] = make_double2(to_double<M>(-(-mm * A1.y + cu * B1u.x - cd * B1d.x) * inva),
                       to_double<M>(-(mm * A1.x + cu * B1u.y - cd * B1d.y) * inva));
  fe[2] = make_double2(to_double<M>((-mm * B1.y - cu * A1u.x + cd * A1d.x) * inva + k * E.x),
                       to_double<M>((mm * B1.x - cu * A1u.y + cd * A1d.y) * inva + k * E.y));
  if (m == 0) { fe[0].y = 0.0; fe[1].y = 0.0; fe[2].y = 0.0; }
}

// F_I = L(state) (+ C(state) when cor.tw != 0) at packed index idx (always double)
__device__ __forceinline__ void linear_point(int m, int n, int T, const double2 *__restrict__ st, int nc, size_t idx,
                                             double inva2, double nu, double phibar, CorArgs cor,
                                             double2 *__restrict__ oI) {
  double2 Phi = st[idx], zeta = st[nc + idx], delta = st[2 * nc + idx];
  if (m == 0) { Phi.y = 0.0; zeta.y = 0.0; delta.y = 0.0; }
  const double k = (double)n * (n + 1) * inva2, nk = nu * k;
  double2 oz = make_double2(-nk * zeta.x, -nk * zeta.y);
  double2 od = make_double2(k * Phi.x - nk * delta.x, k * Phi.y - nk * delta.y);
  if (cor.tw != 0.0) {
    double2 cz, cd;
    coriolis_point(m, n, T, st, nc, idx, cor, &cz, &cd);
    oz.x += cz.x; oz.y += cz.y;
    od.x += cd.x; od.y += cd.y;
  }
  oI[idx] = make_double2(-phibar * delta.x - nk * Phi.x, -phibar * delta.y - nk * Phi.y);
  oI[nc + idx] = oz;
  oI[2 * nc + idx] = od;
}

}  // namespace pfsh
