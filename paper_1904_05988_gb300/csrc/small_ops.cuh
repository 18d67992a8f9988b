// Block-level bodies for one or two states per call, one block per order m:
// velocity recovery + Legendre synthesis, Legendre analysis + assembly of
// F_E and F_I, and the IMEX-SDC node update restricted to the coefficients
// of order m.  Used by the batch-1/2 RHS kernels and by the fused
// single-slice sweep kernel of the PFASST coarse chain (small.cu).
//
// The Legendre rows P_n^m(mu_j), n = m..T+1, of the block's order are staged
// in shared memory once per call with asynchronous copies, at a padded row
// stride (nh + 1) so that lanes that index consecutive degrees hit distinct
// banks (analysis) and lanes that index consecutive latitudes do as well
// (synthesis).  When an order has more rows than the staging buffer holds,
// the rows are processed in chunks.
#pragma once

#include "internal.cuh"
#include "spectral_ops.cuh"

namespace pfsh {

// ---------------------------------------------------------------------------
// asynchronous global -> shared staging (cp.async; every thread of the block
// takes part; completion by stage_wait)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void stage_async(T *dst, const T *src, int n) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const size_t bytes = (size_t)n * sizeof(T);
  if ((((uintptr_t)src | (uintptr_t)d | bytes) & 15) == 0) {
    const char *s8 = reinterpret_cast<const char *>(src);
    for (size_t t = threadIdx.x; t < bytes / 16; t += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + (uint32_t)(16 * t)), "l"(s8 + 16 * t)
                   : "memory");
  } else {
    constexpr int E = (int)sizeof(T);
    static_assert(E == 4 || E == 8 || E == 16, "element size");
    for (int t = threadIdx.x; t < n; t += blockDim.x)
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d + (uint32_t)(E * t)), "l"(src + t), "n"(E)
                   : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// rows [0, nrows) of nh values each -> dst at row stride nh + 1
template <typename R>
__device__ __forceinline__ void stage_rows_async(R *dst, const R *src, int nrows, int nh) {
  constexpr int E = (int)sizeof(R);
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  for (int t = threadIdx.x; t < nrows * nh; t += blockDim.x) {
    const int i = t / nh, j = t - i * nh;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d + (uint32_t)(E * (i * (nh + 1) + j))),
                 "l"(src + t), "n"(E)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void stage_wait() {
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
}

// ---------------------------------------------------------------------------
// shared-memory budgets (bytes); region sizes are rounded to 16 bytes
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <typename R>
__host__ __device__ inline size_t small_stage_bytes(int nlat, int rows) {
  return align16((size_t)rows * (nlat / 2 + 1) * sizeof(R));
}
template <typename R>
__host__ __device__ inline size_t small_synth_work(int T, int nlat, int B, int threads) {
  const int nh = nlat / 2, parts = (threads / nh) > 1 ? threads / nh : 1;
  typedef typename cpx<R>::t C;
  return align16((size_t)(T + 2) * 4 * B * sizeof(C)) + align16((size_t)parts * nh * 2 * 4 * B * sizeof(C));
}
template <typename R>
__host__ __device__ inline size_t small_anal_work(int T, int nlat, int B, int threads) {
  typedef typename cpx<R>::t C;
  const int nh = nlat / 2;
  return align16((size_t)(T + 2) * 5 * B * sizeof(C)) + align16((size_t)2 * nh * 5 * B * sizeof(C)) +
         align16((size_t)threads * 5 * B * sizeof(C));
}
// Largest even row count <= T+2 whose staging fits in `budget` bytes besides
// `fixed` (at least 2).
template <typename R>
__host__ inline int small_stage_rows(size_t fixed, int T, int nlat, size_t budget) {
  const size_t row = (size_t)(nlat / 2 + 1) * sizeof(R);
  long r = budget > fixed + 16 ? (long)((budget - fixed - 16) / row) : 0;
  r = r > T + 2 ? T + 2 : r;
  r &= ~1L;
  return r < 2 ? 2 : (int)r;
}

// ---------------------------------------------------------------------------
// velocity recovery + Legendre synthesis of order m for B <= NB states
//   Pst:   staging buffer of `rows` rows of order m; pmode says who fills the
//          first chunk: STAGE_SELF (this body), STAGE_ISSUED (the caller has
//          issued the copies, this body waits for them) or STAGE_DONE (rows
//          [0, K) are complete, K = T+2-m <= rows required)
//   sm_th: optional shared-memory copy of the state's order-m coefficients
//          ([field][n - m], B = 1); read instead of `state` when given
//   work:  [K][4B] coefficient rows | [parts][nh][2][4B] partial sums
// Called by every thread of a block.
// ---------------------------------------------------------------------------
enum { STAGE_SELF = 0, STAGE_ISSUED = 1, STAGE_DONE = 2 };

template <typename R, int NB>
__device__ __forceinline__ void small_synth_body(int m, int T, int nlat, int B, int rows, R *Pst, int pmode,
                                                 R ma2, R inva, double omega, double phibar, SpecTables<R> tb,
                                                 const R *__restrict__ P, const double2 *__restrict__ state,
                                                 const double2 *sm_th, typename cpx<R>::t *__restrict__ F,
                                                 void *work) {
  typedef typename cpx<R>::t C;
  constexpr int NC = 4 * NB;
  const int nh = nlat / 2, K = T + 2 - m, cols = 4 * B, ld = nh + 1;
  const int parts = max(1, (int)blockDim.x / nh);
  C *Xs = reinterpret_cast<C *>(work);                                               // [K][cols]
  C *Ps = reinterpret_cast<C *>(reinterpret_cast<char *>(work) +
                                align16((size_t)(T + 2) * 4 * B * sizeof(C)));      // [parts][nh][2][cols]
  const int nc = ncoef_of(T);
  const int base = poff(T, m) - m;
  const size_t e0 = (size_t)poff(T + 1, m);
  const R *Pm = P + (size_t)eoff(T, m) * nh;
  // 1. first chunk of Legendre rows in flight while the coefficient rows
  //    (velocity recovery) are computed
  if (pmode == STAGE_SELF) stage_rows_async(Pst, Pm, min(K, rows), nh);
  const int len = T + 1 - m;
  for (int t = threadIdx.x; t < K * B; t += blockDim.x) {
    const int i = t / B, b = t - i * B;
    if (sm_th) {
      prep_point<R>(T, m, m + i, sm_th, sm_th + len, sm_th + 2 * len, -m, e0 + i, tb, ma2, inva, omega, phibar,
                    Xs + (size_t)i * cols);
    } else {
      const double2 *Phi = state + (size_t)b * 3 * nc;
      prep_point<R>(T, m, m + i, Phi, Phi + nc, Phi + 2 * nc, base, e0 + i, tb, ma2, inva, omega, phibar,
                    Xs + (size_t)i * cols + b * 4);
    }
  }
  for (int t = threadIdx.x; t < parts * nh * 2 * cols; t += blockDim.x) Ps[t] = mk<C>(0.0, 0.0);
  if (pmode != STAGE_DONE) stage_wait();
  else __syncthreads();
  // 2. even/odd Legendre sums per latitude; each chunk is split among `parts`
  //    thread groups, partial sums accumulate in Ps
  for (int c0 = 0; c0 < K; c0 += rows) {
    const int cl = min(rows, K - c0);
    const int Kc = ((cl + parts - 1) / parts + 1) & ~1;        // even
    for (int t = threadIdx.x; t < nh * parts; t += blockDim.x) {
      const int j = t % nh, part = t / nh;
      const int i0 = part * Kc, i1 = min(cl, i0 + Kc);
      C e[NC], o[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) e[c] = o[c] = mk<C>(0.0, 0.0);
      for (int i = i0; i < i1; i += 2) {
        const R pe = Pst[(size_t)i * ld + j];
        const bool odd = i + 1 < i1;
        const R po = odd ? Pst[(size_t)(i + 1) * ld + j] : (R)0;
        const C *xe = Xs + (size_t)(c0 + i) * cols, *xo = xe + cols;
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (c < cols) {
            const C u = xe[c];
            e[c].x += pe * u.x;
            e[c].y += pe * u.y;
            if (odd) {
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
          ps[c] = ps[c] + e[c];
          ps[cols + c] = ps[cols + c] + o[c];
        }
    }
    if (c0 + rows < K) {
      __syncthreads();
      stage_rows_async(Pst, Pm + (size_t)(c0 + rows) * nh, min(rows, K - c0 - rows), nh);
      stage_wait();
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
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Legendre analysis of order m + div/curl assembly of F_E and F_I for
// n = m..T, B <= NB states.  Thread groups split the latitudes: thread
// (s, i) sums latitudes [s nh/S, (s+1) nh/S) of degree row i; the S partial
// sums are added in shared memory (no warp-wide butterfly).
//   Pst:  staging buffer of `rows` rows (the first chunk's copies already
//         issued by the caller when p_issued); on return it holds the last
//         chunk (all K rows when K <= rows), so a following synthesis of the
//         same order may reuse it
//   work: [K][5B] analysed rows | [2][nh][5B] hemispheric sums of order m |
//         [threads][5B] partial sums
// Called by every thread of a block.
// ---------------------------------------------------------------------------
template <typename R, int NB>
__device__ __forceinline__ void small_anal_body(int m, int T, int nlat, int B, int rows, R *Pst, bool p_issued,
                                                R inva, R inva2,
                                                double dinva2, double nu, double phibar, CorArgs cor,
                                                const R *__restrict__ eps,
                                                const R *__restrict__ P, const typename cpx<R>::t *__restrict__ H,
                                                const double2 *__restrict__ state, double2 *__restrict__ fE,
                                                double2 *__restrict__ fI, void *work) {
  typedef typename cpx<R>::t C;
  constexpr int NC = 5 * NB;
  const int nh = nlat / 2, K = T + 2 - m, cols = 5 * B, ld = nh + 1;
  char *w = reinterpret_cast<char *>(work);
  C *Ys = reinterpret_cast<C *>(w);                                               // [K][cols]
  w += align16((size_t)(T + 2) * 5 * B * sizeof(C));
  C *Hs = reinterpret_cast<C *>(w);                                               // [2][nh][cols]
  w += align16((size_t)2 * nh * 5 * B * sizeof(C));
  C *Ws = reinterpret_cast<C *>(w);                                               // [threads][cols]
  const R *Pm = P + (size_t)eoff(T, m) * nh;
  stage_async(Hs, H + (size_t)m * 2 * nh * cols, 2 * nh * cols);
  if (!p_issued) stage_rows_async(Pst, Pm, min(K, rows), nh);
  stage_wait();
  // 1. analysis of every degree row of this order
  for (int c0 = 0; c0 < K; c0 += rows) {
    const int cl = min(rows, K - c0);
    const int kw = (cl + 31) & ~31;                                 // rows per latitude group (warp multiple)
    const int S = max(1, min((int)blockDim.x / kw, nh));
    const int t = threadIdx.x, s = t / kw, il = t - s * kw;
    if (s < S && il < cl) {
      const int i = c0 + il, p = i & 1;
      const int j0 = (int)(((long)nh * s) / S), j1 = (int)(((long)nh * (s + 1)) / S);
      const C *h = Hs + (size_t)p * nh * cols;
      const R *pr = Pst + (size_t)il * ld;
      C acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = mk<C>(0.0, 0.0);
      for (int j = j0; j < j1; ++j) {
        const R pv = pr[j];
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
        if (c < cols) Ws[(size_t)t * cols + c] = acc[c];
    }
    __syncthreads();
    for (int u = threadIdx.x; u < cl * cols; u += blockDim.x) {
      const int il2 = u / cols, c = u - il2 * cols;
      C a = mk<C>(0.0, 0.0);
      for (int s2 = 0; s2 < S; ++s2) a = a + Ws[(size_t)(s2 * kw + il2) * cols + c];
      Ys[(size_t)(c0 + il2) * cols + c] = a;
    }
    if (c0 + rows < K) {
      __syncthreads();
      stage_rows_async(Pst, Pm + (size_t)(c0 + rows) * nh, min(rows, K - c0 - rows), nh);
      stage_wait();
    }
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
    if (fI)
      linear_point(m, n, T, state + (size_t)b * 3 * nc, nc, idx, dinva2, nu, phibar, cor, fI + (size_t)b * 3 * nc);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// IMEX-SDC sweep pieces for the coefficients of order m of one state whose
// node arrays are `ns` complex elements apart (Section 5.1.1); the same
// arithmetic as the element-wise sweep kernels.
// ---------------------------------------------------------------------------
// O_i = theta_0 (+ tau_i) + sum_j cE[i][j] F_E,j + cI[i][j] F_I,j, i = 1..M
template <int MAXM>
__device__ __forceinline__ void order_old_part(int m, int T, int M, size_t ns, const SdcCoef &c,
                                               const double2 *__restrict__ th, const double2 *__restrict__ fe,
                                               const double2 *__restrict__ fi, const double2 *__restrict__ tau,
                                               double2 *__restrict__ O) {
  const int nc = ncoef_of(T), p0 = poff(T, m), len = T + 1 - m;
  for (int t = threadIdx.x; t < 3 * len; t += blockDim.x) {
    const int fld = t / len;
    const size_t e = (size_t)fld * nc + p0 + (t - fld * len);
    double2 acc[MAXM + 1];
    const double2 t0 = th[e];
#pragma unroll
    for (int i = 1; i <= MAXM; ++i)
      if (i <= M) acc[i] = tau ? t0 + tau[(size_t)i * ns + e] : t0;
#pragma unroll
    for (int j = 0; j <= MAXM; ++j) {
      if (j > M) break;
      const double2 a = fe[(size_t)j * ns + e], f = fi[(size_t)j * ns + e];
      const double2 sj = make_double2(a.x + f.x, a.y + f.y);
#pragma unroll
      for (int i = 1; i <= MAXM; ++i)
        if (i <= M) {
          if (j == 0 || j > i) {   // cE[i][j] = cI[i][j] = dt Q[i][j] (as in k_sdc_old)
            acc[i].x = fma(c.cE[i][j], sj.x, acc[i].x);
            acc[i].y = fma(c.cE[i][j], sj.y, acc[i].y);
          } else {
            acc[i].x = fma(c.cI[i][j], f.x, fma(c.cE[i][j], a.x, acc[i].x));
            acc[i].y = fma(c.cI[i][j], f.y, fma(c.cE[i][j], a.y, acc[i].y));
          }
        }
    }
#pragma unroll
    for (int i = 1; i <= MAXM; ++i)
      if (i <= M) O[(size_t)(i - 1) * 3 * nc + e] = acc[i];
  }
}

// theta_i = solve(O_i + sum_{1<=j<i} nE[i][j] F_E,j + nI[i][j] F_I,j, h_i)
// with the factors fac[n] of node i (the element-wise kernel k_sdc_node
// documents both layouts: one solve, or two substeps when `split`), also
// written to sm_th[field][n - m] when given
__device__ __forceinline__ void order_node_update(int m, int T, int i, size_t ns, const SdcCoef &c, double hphibar,
                                                  bool split, const double4_32a *__restrict__ fac,
                                                  const double2 *__restrict__ O, const double2 *__restrict__ fe,
                                                  const double2 *__restrict__ fi, double2 *__restrict__ th,
                                                  double2 *sm_th) {
  const int nc = ncoef_of(T), p0 = poff(T, m), len = T + 1 - m;
  double2 *out = th + (size_t)i * ns;
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    const int n = m + t;
    const size_t idx = (size_t)p0 + t;
    double2 r[3];
    for (int f = 0; f < 3; ++f) {
      const size_t e = (size_t)f * nc + idx;
      double2 v = O[e];
      for (int j = 1; j < i; ++j) {
        const double2 a = fe[(size_t)j * ns + e], g = fi[(size_t)j * ns + e];
        v.x = fma(c.nI[i][j], g.x, fma(c.nE[i][j], a.x, v.x));
        v.y = fma(c.nI[i][j], g.y, fma(c.nE[i][j], a.y, v.y));
      }
      r[f] = v;
    }
    const double4_32a q = fac[n];
    double2 x0, x1, x2;
    if (split) {
      double2 old[3];
      for (int f = 0; f < 3; ++f) {
        old[f] = out[(size_t)f * nc + idx];
        r[f].x = fma(-q.z, old[f].x, r[f].x);
        r[f].y = fma(-q.z, old[f].y, r[f].y);
      }
      const double2 y0 = make_double2((r[0].x - hphibar * r[2].x) * q.x, (r[0].y - hphibar * r[2].y) * q.x);
      const double2 y2 = make_double2((r[2].x + q.y * r[0].x) * q.x, (r[2].y + q.y * r[0].y) * q.x);
      x0 = make_double2(fma(q.z, old[0].x, y0.x) * q.w, fma(q.z, old[0].y, y0.y) * q.w);
      x1 = make_double2(fma(q.z, old[1].x, r[1].x) * q.w, fma(q.z, old[1].y, r[1].y) * q.w);
      x2 = make_double2(fma(q.z, old[2].x, y2.x) * q.w, fma(q.z, old[2].y, y2.y) * q.w);
    } else {
      x0 = make_double2((q.x * r[0].x - hphibar * r[2].x) * q.z, (q.x * r[0].y - hphibar * r[2].y) * q.z);
      x1 = make_double2(r[1].x * q.y, r[1].y * q.y);
      x2 = make_double2((q.x * r[2].x + q.w * r[0].x) * q.z, (q.x * r[2].y + q.w * r[0].y) * q.z);
    }
    out[idx] = x0;
    out[nc + idx] = x1;
    out[2 * nc + idx] = x2;
    if (sm_th) {
      sm_th[t] = x0;
      sm_th[len + t] = x1;
      sm_th[2 * len + t] = x2;
    }
  }
}

// The same node update with the Coriolis term implicit: the right-hand sides
// of order m are gathered in sm_th [3][T+1-m] and solved there by the banded
// solve of banded.cuh (scratch: band_scratch_bytes(T) of shared memory; the
// factor table `band` is built with nu = 0 when `split`, and the diffusion
// substep follows as in order_node_update; fac = the node's solve factors).
__device__ __forceinline__ void order_node_update_band(int m, int T, int i, size_t ns, const SdcCoef &c, double h,
                                                       double inva2, double nu, double phibar, bool split,
                                                       CorArgs cor, const double4_32a *__restrict__ band,
                                                       const double4_32a *__restrict__ fac,
                                                       const double2 *__restrict__ O, const double2 *__restrict__ fe,
                                                       const double2 *__restrict__ fi, double2 *__restrict__ th,
                                                       double2 *sm_th, void *scratch) {
  const int nc = ncoef_of(T), p0 = poff(T, m), len = T + 1 - m;
  double2 *out = th + (size_t)i * ns;
  for (int t = threadIdx.x; t < 3 * len; t += blockDim.x) {
    const int f = t / len;
    const size_t e = (size_t)f * nc + p0 + (t - f * len);
    double2 v = O[e];
    for (int j = 1; j < i; ++j) {
      const double2 a = fe[(size_t)j * ns + e], g = fi[(size_t)j * ns + e];
      v.x = fma(c.nI[i][j], g.x, fma(c.nE[i][j], a.x, v.x));
      v.y = fma(c.nI[i][j], g.y, fma(c.nE[i][j], a.y, v.y));
    }
    if (split) {   // r - h nu k old
      const double hnk = fac[m + (t - f * len)].z;
      const double2 o = out[e];
      v.x = fma(-hnk, o.x, v.x);
      v.y = fma(-hnk, o.y, v.y);
    }
    sm_th[t] = v;
  }
  __syncthreads();
  band_order_solve(m, T, h, inva2, split ? 0.0 : nu, phibar, cor, band, fac, split, sm_th, scratch);
  for (int t = threadIdx.x; t < 3 * len; t += blockDim.x) {
    const int f = t / len;
    const size_t e = (size_t)f * nc + p0 + (t - f * len);
    double2 x = sm_th[t];
    if (split) {   // (x* + h nu k old) / s
      const double4_32a q = fac[m + (t - f * len)];
      const double2 o = out[e];
      x = make_double2(fma(q.z, o.x, x.x) * q.w, fma(q.z, o.y, x.y) * q.w);
      sm_th[t] = x;
    }
    out[e] = x;
  }
}

}  // namespace pfsh
