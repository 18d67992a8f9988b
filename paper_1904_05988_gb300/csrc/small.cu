// One or two states per call.
//
// 1. RHS evaluation (swe_rhs and the sweeps with B <= 2): three launches
//    instead of five.
//      k_small_synth  per order m: coefficient rows of eta, Phi', U, V
//                     (velocity recovery of Section 2) in shared memory,
//                     then even/odd Legendre sums at every northern latitude
//                     -> F(+-mu).
//      k_grid_rhs     FFT / grid products / FFT per latitude pair (fft.cu).
//      k_small_anal   per order m: hemispheric sums contracted over latitude,
//                     then the div/curl stencil assembles F_E and F_I.
//
// 2. Step C of Algorithm 1 (the serial coarse chain), one slice after the
//    other.  Everything between two grid stages touches only coefficients of
//    one order m -- the analysis and assembly of node i, the node update and
//    implicit solve of node i+1 (Section 5.1.1), the velocity recovery and
//    synthesis of node i+1 -- so one launch per order does all of it and
//    stages the order's Legendre rows once for both transforms:
//      k_chain_node   [analysis of the previous node] [receive] [old part]
//                     [update + solve of node k] [synthesis of node k]
//    A slice's sweep is then k_chain_node / k_grid_rhs pairs, one per node.
//    The right-hand side of the received value (node 0 of slice n) is the
//    right-hand side the sender evaluated at its last node: the same state
//    through the same kernels, so it is copied with the state instead of
//    being evaluated again.
//
// The arithmetic is that of the batched path's kernels, in the plan's real
// type for the contractions (fp64 for FP64 plans, fp32 otherwise) and fp64
// for the spectral parts.
#include "internal.cuh"
#include "small_ops.cuh"
#include "spectral_ops.cuh"

namespace pfsh {

constexpr int kSmallMaxStates = 2;
constexpr int kSynthThreads = 256, kAnalThreads = 512, kChainThreads = 512;
constexpr size_t kStageBudget = 100 * 1024;   // two blocks per SM
constexpr size_t kChainBudget = 200 * 1024;   // one block per SM

template <typename R, int NB>
__global__ void __launch_bounds__(kSynthThreads) k_small_synth(int T, int nlat, int B, int rows, R ma2, R inva,
                                                               double omega, double phibar, SpecTables<R> tb,
                                                               const R *__restrict__ P,
                                                               const double2 *__restrict__ state,
                                                               typename cpx<R>::t *__restrict__ F) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *Pst = reinterpret_cast<R *>(smem_raw);
  small_synth_body<R, NB>(blockIdx.x, T, nlat, B, rows, Pst, STAGE_SELF, ma2, inva, omega, phibar, tb, P, state,
                          nullptr, F, smem_raw + small_stage_bytes<R>(nlat, rows));
}

template <typename R, int NB>
__global__ void __launch_bounds__(kAnalThreads) k_small_anal(int T, int nlat, int B, int rows, R inva, R inva2,
                                                             double dinva2, double nu, double phibar, CorArgs cor,
                                                             const R *__restrict__ eps, const R *__restrict__ P,
                                                             const typename cpx<R>::t *__restrict__ H,
                                                             const double2 *__restrict__ state,
                                                             double2 *__restrict__ fE, double2 *__restrict__ fI) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *Pst = reinterpret_cast<R *>(smem_raw);
  small_anal_body<R, NB>(blockIdx.x, T, nlat, B, rows, Pst, false, inva, inva2, dinva2, nu, phibar, cor, eps, P, H,
                         state, fE, fI, smem_raw + small_stage_bytes<R>(nlat, rows));
}

template <typename R, int NB>
static int small_launch(const sht_plan *p, const double *state, double *fE, double *fI, int B, const swe_params &prm,
                        CorArgs cor, const R *P, SpecTables<R> tb, cudaStream_t s) {
  typedef typename cpx<R>::t C;
  const int T = p->T, nlat = p->nlat;
  const size_t w1 = small_synth_work<R>(T, nlat, B, kSynthThreads);
  const int r1 = small_stage_rows<R>(w1, T, nlat, kStageBudget);
  const size_t sm1 = w1 + small_stage_bytes<R>(nlat, r1);
  int rc = ensure_smem((const void *)k_small_synth<R, NB>, sm1);
  if (rc) return rc;
  {
    PFSH_LAUNCH("k_small_synth", s);
    k_small_synth<R, NB><<<T + 1, kSynthThreads, sm1, s>>>(T, nlat, B, r1, (R)(-prm.a * prm.a), (R)(1.0 / prm.a),
                                                           omega_explicit(prm), prm.phibar, tb, P,
                                                           (const double2 *)state, (C *)p->F);
  }
  PFSH_CHECK_LAUNCH("k_small_synth");
  if ((rc = grid_rhs(p, B, prm, s))) return rc;
  const size_t w3 = small_anal_work<R>(T, nlat, B, kAnalThreads);
  const int r3 = small_stage_rows<R>(w3, T, nlat, kStageBudget);
  const size_t sm3 = w3 + small_stage_bytes<R>(nlat, r3);
  if ((rc = ensure_smem((const void *)k_small_anal<R, NB>, sm3))) return rc;
  const double inva2 = 1.0 / (prm.a * prm.a);
  {
    PFSH_LAUNCH("k_small_anal", s);
    k_small_anal<R, NB><<<T + 1, kAnalThreads, sm3, s>>>(T, nlat, B, r3, (R)(1.0 / prm.a), (R)inva2, inva2,
                                                         prm.nu, prm.phibar, cor, tb.eps, P, (const C *)p->H,
                                                         (const double2 *)state, (double2 *)fE, (double2 *)fI);
  }
  PFSH_CHECK_LAUNCH("k_small_anal");
  return PFSH_OK;
}

bool small_rhs(int B) { return B <= kSmallMaxStates; }

int rhs_small(const sht_plan *p, const double *state, double *fE, double *fI, int B, const swe_params &prm,
              CorArgs cor, cudaStream_t s) {
  const SpecTables<double> t64{p->d_eps, p->d_ilap};
  const SpecTables<float> t32{p->d_eps32, p->d_ilap32};
  if (p->prec == PFSH_FP64)
    return B == 1 ? small_launch<double, 1>(p, state, fE, fI, B, prm, cor, p->d_P, t64, s)
                  : small_launch<double, 2>(p, state, fE, fI, B, prm, cor, p->d_P, t64, s);
  return B == 1 ? small_launch<float, 1>(p, state, fE, fI, B, prm, cor, p->d_P32, t32, s)
                : small_launch<float, 2>(p, state, fE, fI, B, prm, cor, p->d_P32, t32, s);
}

// ---------------------------------------------------------------------------
// fused single-slice sweep step (Step C)
// ---------------------------------------------------------------------------
struct ChainStep {
  // analysis + assembly of one node: its state (for F_I) and outputs
  const double2 *a_th;        // nullptr: no analysis in this launch
  double2 *a_fe, *a_fi;
  // receive: copy theta, F_E, F_I of (slice n-1, last node) to (slice n, node 0)
  const double2 *r_th, *r_fe, *r_fi;   // nullptr: no receive
  // sweep of one slice: node 0 at th/fe/fi, nodes ns complex apart
  double2 *th, *fe, *fi;
  const double2 *tau;         // FAS term of the slice (node 0), nullable
  double2 *O;                 // [M][3 nc] old parts
  size_t ns;
  int k, M;                   // node to update (0: none) and last node
  double hphibar;             // dt QI[k][k] Phibar
  const double4_32a *fac;     // solve factors of node k [T+1]
  double h;                   // dt QI[k][k]
  const double4_32a *band;    // Coriolis implicit: banded-solve factors of node k [2][nc]
};

template <typename R>
struct ChainGeo {
  int T, nlat, rows;
  size_t work;                // bytes of the body work region
  R ma2, inva, inva2;
  double dinva2, omega, nu, phibar;
  bool split;                 // two-substep node solve
  CorArgs cor;
  SpecTables<R> tb;
  const R *P;
  typename cpx<R>::t *F;
  const typename cpx<R>::t *H;
};

// At most 64 registers per thread (two blocks' worth per SM): a launch of this
// kernel is latency-bound and holds one SM per order, and with the register
// file half free the fine-sweep kernels of the other stream (grid stage,
// synthesis) can run on the same SMs meanwhile (measured: 188 -> 197
// iterations/s at T255/T127 with 32 slices, despite some spilling).
template <typename R>
__global__ void __launch_bounds__(kChainThreads, 2) k_chain_node(ChainStep st, ChainGeo<R> g, SdcCoef c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = blockIdx.x, T = g.T, nc = ncoef_of(T), K = T + 2 - m;
  R *Pst = reinterpret_cast<R *>(smem_raw);
  unsigned char *work = smem_raw + small_stage_bytes<R>(g.nlat, g.rows);
  double2 *thk = reinterpret_cast<double2 *>(work + g.work);   // [3][T+1-m] state of node k, order m
  const bool anal = st.a_th != nullptr;
  // independent prologue: the order's Legendre rows (a table), then wait for
  // the previous kernel of the stream (programmatic dependent launch)
  stage_rows_async(Pst, g.P + (size_t)eoff(T, m) * (g.nlat / 2), min(K, g.rows), g.nlat / 2);
  pdl_wait();
  if (anal)
    small_anal_body<R, 1>(m, T, g.nlat, 1, g.rows, Pst, true, g.inva, g.inva2, g.dinva2, g.nu, g.phibar, g.cor,
                          g.tb.eps,
                          g.P, g.H, st.a_th, st.a_fe, st.a_fi, work);
  if (st.k == 0) {
    if (!anal) stage_wait();
    return;
  }
  const int p0 = poff(T, m), len = T + 1 - m;
  if (st.r_th) {
    for (int t = threadIdx.x; t < 3 * len; t += blockDim.x) {
      const int fld = t / len;
      const size_t e = (size_t)fld * nc + p0 + (t - fld * len);
      st.th[e] = st.r_th[e];
      st.fe[e] = st.r_fe[e];
      st.fi[e] = st.r_fi[e];
    }
    __syncthreads();
  }
  if (st.k == 1) {
    order_old_part<8>(m, T, st.M, st.ns, c, st.th, st.fe, st.fi, st.tau, st.O);
    __syncthreads();
  }
  if (g.cor.tw != 0.0)   // the analysis is done: its work region holds the banded solve's scratch
    order_node_update_band(m, T, st.k, st.ns, c, st.h, g.dinva2, g.nu, g.phibar, g.split, g.cor, st.band, st.fac,
                           st.O + (size_t)(st.k - 1) * 3 * nc, st.fe, st.fi, st.th, thk, work);
  else
    order_node_update(m, T, st.k, st.ns, c, st.hphibar, g.split, st.fac, st.O + (size_t)(st.k - 1) * 3 * nc, st.fe,
                      st.fi, st.th, thk);
  __syncthreads();
  // rows issued in the prologue: complete after the analysis, else in flight
  const int pmode = anal ? (K <= g.rows ? STAGE_DONE : STAGE_SELF) : STAGE_ISSUED;
  small_synth_body<R, 1>(m, T, g.nlat, 1, g.rows, Pst, pmode, g.ma2, g.inva, g.omega, g.phibar, g.tb, g.P,
                         st.th + (size_t)st.k * st.ns, thk, g.F, work);
}

template <typename R>
static int chain_node_launch(const ChainStep &st, ChainGeo<R> g, const SdcCoef &c, cudaStream_t s, bool pdl) {
  g.work = std::max(small_synth_work<R>(g.T, g.nlat, 1, kChainThreads),
                    small_anal_work<R>(g.T, g.nlat, 1, kChainThreads));
  if (g.cor.tw != 0.0) g.work = std::max(g.work, align16(band_scratch_bytes(g.T)));
  const size_t thk = align16((size_t)3 * (g.T + 1) * sizeof(double2));
  g.rows = small_stage_rows<R>(g.work + thk, g.T, g.nlat, kChainBudget);
  const size_t smem = g.work + thk + small_stage_bytes<R>(g.nlat, g.rows);
  int rc = ensure_smem((const void *)k_chain_node<R>, smem);
  if (rc) return rc;
  {
    PFSH_LAUNCH("k_chain_node", s);
    if (pdl) {
      cudaError_t e = launch_pdl(k_chain_node<R>, dim3(g.T + 1), dim3(kChainThreads), smem, s, st, g, c);
      if (e != cudaSuccess) return cuda_fail(e, "k_chain_node");
    } else {
      k_chain_node<R><<<g.T + 1, kChainThreads, smem, s>>>(st, g, c);
    }
  }
  PFSH_CHECK_LAUNCH("k_chain_node");
  return PFSH_OK;
}

// ---------------------------------------------------------------------------
// Step C with the low orders shared by two blocks
// ---------------------------------------------------------------------------
// The block of order m does work in proportion to the K = T + 2 - m degree
// rows n = m..T+1 of the order, so a launch lasts as long as the low orders.
// Orders m < msplit are therefore shared by two blocks: part 0 owns the rows
// i = n - m in [0, h), part 1 the rows in [h, K) (h even, about K/2).  Each
// block computes what its own rows need: the analysed rows of the previous
// node for [i0 - 2, i1 + 2) (the assembly of row i reads rows i +- 1), F_E and
// F_I for [i0 - 1, i1 + 1), the node update for the same rows (the velocity
// recovery of row i reads the stream function and velocity potential at
// i +- 1), and the synthesis sums over its own rows only, into F (part 0) or
// F2 (part 1), which the grid stage adds.  Both blocks compute the shared
// halo rows the same way (each row's latitude sum is split into the same
// segments in every block of a launch) and each stores only its own rows.
// The node-0 values of a slice that receives are read from the sender's
// arrays (global) or, for F_E and F_I of the node analysed in the same
// launch, from shared memory, never from locations another block writes in
// the same launch.  Used for the one-solve node update with the Coriolis term
// explicit (the banded solve couples all degrees of an order, and the
// two-substep solve reads the node's old iterate, which the other block of
// the order overwrites).
struct ChainRange {
  int m, part, K;
  int i0, i1;   // own rows
  int u0, u1;   // rows whose F_E, F_I and updated state the block needs (coefficient rows, i <= K - 2)
  int a0, a1;   // analysed rows
};

__host__ __device__ inline int chain_split_point(int K) { return ((K + 1) / 2 + 1) & ~1; }

__host__ __device__ inline ChainRange chain_range(int T, int msplit, int bid) {
  ChainRange r;
  r.m = bid <= T ? bid : bid - (T + 1);
  r.part = bid <= T ? 0 : 1;
  r.K = T + 2 - r.m;
  if (r.m < msplit) {
    const int h = chain_split_point(r.K);
    r.i0 = r.part ? h : 0;
    r.i1 = r.part ? r.K : h;
  } else {
    r.i0 = 0;
    r.i1 = r.K;
  }
  r.u0 = r.i0 > 0 ? r.i0 - 1 : 0;
  r.u1 = r.i1 + 1 < r.K - 1 ? r.i1 + 1 : r.K - 1;
  r.a0 = r.u0 > 0 ? r.u0 - 1 : 0;
  r.a1 = r.u1 + 1 < r.K ? r.u1 + 1 : r.K;
  return r;
}

template <typename R>
struct SplitGeo {
  int T, nlat, msplit;
  int rows;          // Legendre rows staged at once (even)
  int kw, S;         // analysis: rows per latitude group, latitude segments (fixed per launch)
  int UL;            // stride of the per-block coefficient-row arrays (>= max u1 - u0)
  int YL;            // rows of the analysed-row array (>= max a1 - a0)
  int XL;            // rows of the synthesis input array (>= max i1 - i0)
  size_t o_work, o_per;   // byte offsets: work region (union of analysis / synthesis), persistent arrays
  R ma2, inva, inva2;
  double dinva2, omega, nu, phibar;
  SpecTables<R> tb;
  const R *P;
  typename cpx<R>::t *F, *F2;
  const typename cpx<R>::t *H;
};

template <typename R>
__global__ void __launch_bounds__(kChainThreads, 2) k_chain_split(ChainStep st, SplitGeo<R> g, SdcCoef c) {
  typedef typename cpx<R>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int T = g.T, nlat = g.nlat, nh = nlat / 2, ld = nh + 1, nc = ncoef_of(T);
  const ChainRange rg = chain_range(T, g.msplit, blockIdx.x);
  const int m = rg.m, UL = g.UL;
  R *Pst = reinterpret_cast<R *>(smem_raw);
  unsigned char *work = smem_raw + g.o_work;
  double2 *per = reinterpret_cast<double2 *>(smem_raw + g.o_per);
  double2 *feS = per, *fiS = per + 3 * UL, *O1S = per + 6 * UL, *thk = per + 9 * UL;   // [3][UL] each
  const bool anal = st.a_th != nullptr;
  const R *Pm = g.P + (size_t)eoff(T, m) * nh;
  const int p0 = poff(T, m);
  const size_t e0 = (size_t)poff(T + 1, m);   // extended-triangle row of (m, m)
  // independent prologue: the first rows this block reads
  const int s0 = anal ? rg.a0 : rg.i0, s1 = anal ? rg.a1 : rg.i1;
  stage_rows_async(Pst, Pm + (size_t)s0 * nh, min(g.rows, s1 - s0), nh);
  pdl_wait();
  bool staged_all = s1 - s0 <= g.rows;   // Pst holds rows [s0, s1)
  if (anal) {
    // 1. analysis of rows [a0, a1) of the node st.a_th
    C *Ys = reinterpret_cast<C *>(work);                                   // [YL][5]
    C *Hs = Ys + (size_t)g.YL * 5;                                         // [2][nh][5]
    C *Ws = Hs + (size_t)2 * nh * 5;                                       // [threads][5]
    stage_async(Hs, g.H + (size_t)m * 2 * nh * 5, 2 * nh * 5);
    for (int c0 = rg.a0; c0 < rg.a1; c0 += g.rows) {
      const int cl = min(g.rows, rg.a1 - c0);
      if (c0 != rg.a0) {
        __syncthreads();
        stage_rows_async(Pst, Pm + (size_t)c0 * nh, cl, nh);
      }
      stage_wait();
      const int t = threadIdx.x, s = t / g.kw, il = t - s * g.kw;
      if (s < g.S && il < cl) {
        const int i = c0 + il, par = i & 1;
        const int j0 = (int)(((long)nh * s) / g.S), j1 = (int)(((long)nh * (s + 1)) / g.S);
        const C *h = Hs + (size_t)par * nh * 5;
        const R *pr = Pst + (size_t)il * ld;
        C acc[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) acc[f] = mk<C>(0.0, 0.0);
        for (int j = j0; j < j1; ++j) {
          const R pv = pr[j];
#pragma unroll
          for (int f = 0; f < 5; ++f) {
            const C v = h[(size_t)j * 5 + f];
            acc[f].x += pv * v.x;
            acc[f].y += pv * v.y;
          }
        }
#pragma unroll
        for (int f = 0; f < 5; ++f) Ws[(size_t)t * 5 + f] = acc[f];
      }
      __syncthreads();
      for (int u = threadIdx.x; u < cl * 5; u += blockDim.x) {
        const int il2 = u / 5, f = u - il2 * 5;
        C a = mk<C>(0.0, 0.0);
        for (int s2 = 0; s2 < g.S; ++s2) a = a + Ws[(size_t)(s2 * g.kw + il2) * 5 + f];
        Ys[(size_t)(c0 - rg.a0 + il2) * 5 + f] = a;
      }
    }
    __syncthreads();
    // 2. F_E and F_I of rows [u0, u1) (shared memory), own rows also stored
    for (int t = threadIdx.x; t < rg.u1 - rg.u0; t += blockDim.x) {
      const int i = rg.u0 + t, n = m + i;
      C cur[5], up[5], dn[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        cur[f] = Ys[(size_t)(i - rg.a0) * 5 + f];
        up[f] = Ys[(size_t)(i + 1 - rg.a0) * 5 + f];
        dn[f] = i ? Ys[(size_t)(i - 1 - rg.a0) * 5 + f] : mk<C>(0.0, 0.0);
      }
      double2 fe[3], fi[3];
      assemble_point<R, C>(m, n, cur, up, dn, i > 0, g.tb.eps[e0 + i + 1], g.tb.eps[e0 + i], g.inva, g.inva2, fe);
      const size_t idx = (size_t)p0 + i;
      linear_vals(m, n, T, st.a_th, nc, idx, g.dinva2, g.nu, g.phibar, CorArgs{nullptr, 0.0}, fi);
      const bool own = i >= rg.i0 && i < rg.i1;
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        feS[f * UL + t] = fe[f];
        fiS[f * UL + t] = fi[f];
        if (own) {
          st.a_fe[(size_t)f * nc + idx] = fe[f];
          st.a_fi[(size_t)f * nc + idx] = fi[f];
        }
      }
    }
    __syncthreads();
    staged_all = rg.a1 - rg.a0 <= g.rows;   // rows [a0, a1) are all in Pst
  }
  if (st.k == 0) {
    if (!anal) stage_wait();
    return;
  }
  const int K1 = rg.K - 1;   // coefficient rows i < K1 (n <= T)
  const int c0r = rg.i0, c1r = min(rg.i1, K1);   // own coefficient rows
  // 3. receive: own coefficient rows of node 0 from the sender's last node
  if (st.r_th) {
    for (int t = threadIdx.x; t < 3 * (c1r - c0r); t += blockDim.x) {
      const int f = t / (c1r - c0r);
      const size_t e = (size_t)f * nc + p0 + c0r + (t - f * (c1r - c0r));
      st.th[e] = st.r_th[e];
      st.fe[e] = st.r_fe[e];
      st.fi[e] = st.r_fi[e];
    }
  }
  const int M = st.M, k = st.k;
  // node-0 sources for this launch (never a location another block writes now)
  const double2 *th0 = st.r_th ? st.r_th : st.th;
  const double2 *fe0 = st.r_fe ? st.r_fe : st.fe;
  const double2 *fi0 = st.r_fi ? st.r_fi : st.fi;
  // 4. old parts O_i (i = 1..M) of rows [u0, u1) at the first node; own rows stored
  if (k == 1) {
    for (int t = threadIdx.x; t < 3 * (rg.u1 - rg.u0); t += blockDim.x) {
      const int f = t / (rg.u1 - rg.u0), tt = t - f * (rg.u1 - rg.u0), i = rg.u0 + tt;
      const size_t e = (size_t)f * nc + p0 + i;
      double2 acc[9];
      const double2 t0 = th0[e];
#pragma unroll
      for (int q = 1; q <= 8; ++q)
        if (q <= M) acc[q] = st.tau ? t0 + st.tau[(size_t)q * st.ns + e] : t0;
#pragma unroll
      for (int j = 0; j <= 8; ++j) {
        if (j > M) break;
        double2 a, fv;
        if (j == 0) {
          a = anal ? feS[f * UL + tt] : fe0[e];
          fv = anal ? fiS[f * UL + tt] : fi0[e];
        } else {
          a = st.fe[(size_t)j * st.ns + e];
          fv = st.fi[(size_t)j * st.ns + e];
        }
        const double2 sj = make_double2(a.x + fv.x, a.y + fv.y);
#pragma unroll
        for (int q = 1; q <= 8; ++q)
          if (q <= M) {
            if (j == 0 || j > q) {
              acc[q].x = fma(c.cE[q][j], sj.x, acc[q].x);
              acc[q].y = fma(c.cE[q][j], sj.y, acc[q].y);
            } else {
              acc[q].x = fma(c.cI[q][j], fv.x, fma(c.cE[q][j], a.x, acc[q].x));
              acc[q].y = fma(c.cI[q][j], fv.y, fma(c.cE[q][j], a.y, acc[q].y));
            }
          }
      }
      O1S[f * UL + tt] = acc[1];
      if (i >= c0r && i < c1r)
#pragma unroll
        for (int q = 1; q <= 8; ++q)
          if (q <= M) st.O[(size_t)(q - 1) * 3 * nc + e] = acc[q];
    }
    __syncthreads();
  }
  // 5. node update of node k for rows [u0, u1): one solve per coefficient
  for (int tt = threadIdx.x; tt < rg.u1 - rg.u0; tt += blockDim.x) {
    const int i = rg.u0 + tt, n = m + i;
    const size_t idx = (size_t)p0 + i;
    double2 r[3];
    for (int f = 0; f < 3; ++f) {
      const size_t e = (size_t)f * nc + idx;
      double2 v = k == 1 ? O1S[f * UL + tt] : st.O[(size_t)(k - 1) * 3 * nc + e];
      for (int j = 1; j < k; ++j) {
        const bool here = anal && j == k - 1;
        const double2 a = here ? feS[f * UL + tt] : st.fe[(size_t)j * st.ns + e];
        const double2 gi = here ? fiS[f * UL + tt] : st.fi[(size_t)j * st.ns + e];
        v.x = fma(c.nI[k][j], gi.x, fma(c.nE[k][j], a.x, v.x));
        v.y = fma(c.nI[k][j], gi.y, fma(c.nE[k][j], a.y, v.y));
      }
      r[f] = v;
    }
    const double4_32a q = st.fac[n];
    const double2 x0 = make_double2((q.x * r[0].x - st.hphibar * r[2].x) * q.z, (q.x * r[0].y - st.hphibar * r[2].y) * q.z);
    const double2 x1 = make_double2(r[1].x * q.y, r[1].y * q.y);
    const double2 x2 = make_double2((q.x * r[2].x + q.w * r[0].x) * q.z, (q.x * r[2].y + q.w * r[0].y) * q.z);
    thk[tt] = x0;
    thk[UL + tt] = x1;
    thk[2 * UL + tt] = x2;
    if (i >= c0r && i < c1r) {
      double2 *out = st.th + (size_t)k * st.ns;
      out[idx] = x0;
      out[nc + idx] = x1;
      out[2 * nc + idx] = x2;
    }
  }
  __syncthreads();
  // 6. velocity recovery of the own rows and their synthesis sums
  C *Xs = reinterpret_cast<C *>(work);                                      // [XL][4]
  const int parts = max(1, (int)blockDim.x / nh);
  C *Ps = Xs + (size_t)g.XL * 4;                                            // [parts][nh][2][4]
  const int nown = rg.i1 - rg.i0;
  for (int t = threadIdx.x; t < nown; t += blockDim.x) {
    const int i = rg.i0 + t;
    prep_point<R>(T, m, m + i, thk, thk + UL, thk + 2 * UL, -m - rg.u0, e0 + i, g.tb, g.ma2, g.inva, g.omega,
                  g.phibar, Xs + (size_t)t * 4);
  }
  for (int t = threadIdx.x; t < parts * nh * 2 * 4; t += blockDim.x) Ps[t] = mk<C>(0.0, 0.0);
  // rows [i0, i1) in Pst: reuse the analysis staging when it holds them, else stage
  int pbase;   // row of Pst[0]
  if (!anal) {
    stage_wait();   // prologue rows [i0, ...)
    pbase = rg.i0;
  } else if (staged_all) {
    __syncthreads();
    pbase = rg.a0;
  } else {
    __syncthreads();
    stage_rows_async(Pst, Pm + (size_t)rg.i0 * nh, min(g.rows, nown), nh);
    stage_wait();
    pbase = rg.i0;
  }
  for (int c0 = 0; c0 < nown; c0 += g.rows) {
    const int cl = min(g.rows, nown - c0);
    if (c0 > 0) {
      __syncthreads();
      stage_rows_async(Pst, Pm + (size_t)(rg.i0 + c0) * nh, cl, nh);
      stage_wait();
      pbase = rg.i0 + c0;
    }
    const int Kc = ((cl + parts - 1) / parts + 1) & ~1;   // even
    for (int t = threadIdx.x; t < nh * parts; t += blockDim.x) {
      const int j = t % nh, pp = t / nh;
      const int q0 = pp * Kc, q1 = min(cl, q0 + Kc);
      C e[4], o[4];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) e[cc] = o[cc] = mk<C>(0.0, 0.0);
      for (int q = q0; q < q1; q += 2) {
        const int i = rg.i0 + c0 + q;              // even relative to the order's first row
        const R pe = Pst[(size_t)(i - pbase) * ld + j];
        const bool odd = q + 1 < q1;
        const R po = odd ? Pst[(size_t)(i + 1 - pbase) * ld + j] : (R)0;
        const C *xe = Xs + (size_t)(c0 + q) * 4, *xo = xe + 4;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const C u = xe[cc];
          e[cc].x += pe * u.x;
          e[cc].y += pe * u.y;
          if (odd) {
            const C v = xo[cc];
            o[cc].x += po * v.x;
            o[cc].y += po * v.y;
          }
        }
      }
      C *ps = Ps + ((size_t)pp * nh + j) * 8;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        ps[cc] = ps[cc] + e[cc];
        ps[4 + cc] = ps[4 + cc] + o[cc];
      }
    }
  }
  __syncthreads();
  C *Fo = rg.part ? g.F2 : g.F;
  for (int t = threadIdx.x; t < nh * 4; t += blockDim.x) {
    const int j = t / 4, cc = t - j * 4;
    C E = mk<C>(0.0, 0.0), O = mk<C>(0.0, 0.0);
    for (int pp = 0; pp < parts; ++pp) {
      const C *ps = Ps + ((size_t)pp * nh + j) * 8;
      E = E + ps[cc];
      O = O + ps[4 + cc];
    }
    Fo[((size_t)m * nlat + j) * 4 + cc] = E + O;
    Fo[((size_t)m * nlat + (nlat - 1 - j)) * 4 + cc] = E - O;
  }
}

// launch geometry of k_chain_split: per-block ranges, staging rows, offsets
template <typename R>
static SplitGeo<R> split_geo(const ChainGeo<R> &cg, const sht_plan *p, size_t budget) {
  typedef typename cpx<R>::t C;
  SplitGeo<R> g{};
  const int T = cg.T, nh = cg.nlat / 2;
  g.T = T;
  g.nlat = cg.nlat;
  // orders with more rows than about half of order 0's are shared by two blocks
  int ms = 0;
  while (ms <= T && T + 2 - ms > (T + 2) / 2 + 2) ++ms;
  g.msplit = ms;
  int UL = 0, YL = 0, XL = 0;
  for (int b = 0; b < T + 1 + ms; ++b) {
    const ChainRange r = chain_range(T, ms, b);
    UL = std::max(UL, r.u1 - r.u0);
    YL = std::max(YL, r.a1 - r.a0);
    XL = std::max(XL, r.i1 - r.i0);
  }
  g.UL = std::max(UL, 1);
  g.YL = YL;
  g.XL = XL;
  const int parts = std::max(1, kChainThreads / nh);
  const size_t per = align16((size_t)12 * g.UL * sizeof(double2));
  const size_t w_an = align16((size_t)g.YL * 5 * sizeof(C)) + align16((size_t)2 * nh * 5 * sizeof(C)) +
                      align16((size_t)kChainThreads * 5 * sizeof(C));
  const size_t w_sy = align16((size_t)g.XL * 4 * sizeof(C)) + align16((size_t)parts * nh * 2 * 4 * sizeof(C));
  const size_t w = std::max(w_an, w_sy);
  g.rows = small_stage_rows<R>(w + per, T, cg.nlat, budget);
  g.rows = std::min(g.rows, (YL + 1) & ~1);
  if (g.rows < 2) g.rows = 2;
  g.o_work = small_stage_bytes<R>(cg.nlat, g.rows);
  g.o_per = g.o_work + w;
  g.kw = (std::min(g.rows, YL) + 31) & ~31;
  g.S = std::max(1, std::min(kChainThreads / g.kw, nh));
  g.ma2 = cg.ma2;
  g.inva = cg.inva;
  g.inva2 = cg.inva2;
  g.dinva2 = cg.dinva2;
  g.omega = cg.omega;
  g.nu = cg.nu;
  g.phibar = cg.phibar;
  g.tb = cg.tb;
  g.P = cg.P;
  g.F = cg.F;
  g.F2 = (C *)p->F2;
  g.H = cg.H;
  return g;
}

template <typename R>
static size_t split_smem(const SplitGeo<R> &g) {
  return g.o_per + align16((size_t)12 * g.UL * sizeof(double2));
}

template <typename R>
static int chain_split_launch(const ChainStep &st, const SplitGeo<R> &g, const SdcCoef &c, cudaStream_t s,
                              bool pdl) {
  const size_t smem = split_smem(g);
  int rc = ensure_smem((const void *)k_chain_split<R>, smem);
  if (rc) return rc;
  const int blocks = g.T + 1 + g.msplit;
  {
    PFSH_LAUNCH("k_chain_node", s);
    if (pdl) {
      cudaError_t e = launch_pdl(k_chain_split<R>, dim3(blocks), dim3(kChainThreads), smem, s, st, g, c);
      if (e != cudaSuccess) return cuda_fail(e, "k_chain_node");
    } else {
      k_chain_split<R><<<blocks, kChainThreads, smem, s>>>(st, g, c);
    }
  }
  PFSH_CHECK_LAUNCH("k_chain_node");
  return PFSH_OK;
}

template <typename R>
static ChainGeo<R> chain_geo(const swe_ctx *ctx, const R *P, SpecTables<R> tb) {
  typedef typename cpx<R>::t C;
  const sht_plan *p = ctx->plan;
  const swe_params &prm = ctx->prm;
  const double inva2 = 1.0 / (prm.a * prm.a);
  return ChainGeo<R>{p->T, p->nlat, 0, 0, (R)(-prm.a * prm.a), (R)(1.0 / prm.a), (R)inva2, inva2, omega_explicit(prm),
                     prm.nu, prm.phibar, prm.implicit_split != 0, cor_args(ctx), tb, P, (C *)p->F, (const C *)p->H};
}

template <typename R>
static int chain_typed(sdc_level *l, ChainGeo<R> g, double *th, double *fe, double *fi, const double *tau,
                       size_t node_stride, size_t slice_stride, int n0, int n1, bool recv_first, cudaStream_t s,
                       cudaEvent_t after_first) {
  const swe_ctx *ctx = l->ctx;
  const sht_plan *p = ctx->plan;
  const int M = l->nodes - 1;
  const SdcCoef c = sdc_coef(l);
  const size_t ns = node_stride / 2, ss = slice_stride / 2;
  double2 *TH = (double2 *)th, *FE = (double2 *)fe, *FI = (double2 *)fi;
  const double2 *TAU = (const double2 *)tau;
  int rc;
  // the low orders shared by two blocks: one-solve node update, Coriolis term explicit
  const bool split = p->F2 && !g.split && g.cor.tw == 0.0;
  SplitGeo<R> sg{};
  if (split) sg = split_geo<R>(g, p, kChainBudget);
  const int msplit = split ? sg.msplit : 0;
  auto step = [&](const ChainStep &cs, bool pdl) {
    return split ? chain_split_launch<R>(cs, sg, c, s, pdl) : chain_node_launch<R>(cs, g, c, s, pdl);
  };
  for (int n = n0; n < n1; ++n) {
    for (int k = 1; k <= M; ++k) {
      ChainStep st = {};
      st.th = TH + n * ss;
      st.fe = FE + n * ss;
      st.fi = FI + n * ss;
      st.tau = TAU ? TAU + n * ss : nullptr;
      st.O = (double2 *)l->d_old;
      st.ns = ns;
      st.k = k;
      st.M = M;
      st.hphibar = c.h[k] * ctx->prm.phibar;
      st.fac = (const double4_32a *)l->d_fac + (size_t)k * (p->T + 1);
      st.h = c.h[k];
      st.band = l->d_band ? l->d_band + (size_t)k * band_table_entries(p->ncoef) : nullptr;
      const bool recv = k == 1 && (n > n0 || recv_first);
      if (k > 1) {                                   // analysis of node k-1 of this slice
        st.a_th = st.th + (k - 1) * ns;
        st.a_fe = st.fe + (k - 1) * ns;
        st.a_fi = st.fi + (k - 1) * ns;
      } else if (n > n0) {                           // analysis of the sender's last node
        st.a_th = TH + (n - 1) * ss + M * ns;
        st.a_fe = FE + (n - 1) * ss + M * ns;
        st.a_fi = FI + (n - 1) * ss + M * ns;
      }
      if (recv) {
        st.r_th = TH + (n - 1) * ss + M * ns;
        st.r_fe = FE + (n - 1) * ss + M * ns;
        st.r_fi = FI + (n - 1) * ss + M * ns;
      }
      // the first launch of the chain follows other work of the stream
      if ((rc = step(st, n > n0 || k > 1))) return rc;
      if (after_first && n == n0 && k == 1) PFSH_CUDA(cudaEventRecord(after_first, s));
      if ((rc = grid_rhs(p, 1, ctx->prm, s, true, msplit))) return rc;
    }
  }
  if (n1 > n0) {   // analysis of the last slice's last node
    ChainStep st = {};
    st.a_th = TH + (n1 - 1) * ss + M * ns;
    st.a_fe = FE + (n1 - 1) * ss + M * ns;
    st.a_fi = FI + (n1 - 1) * ss + M * ns;
    if ((rc = step(st, true))) return rc;
  }
  return PFSH_OK;
}

int chain_prepare(sht_plan *p) {
  if (p->F2) return PFSH_OK;
  const size_t bytes = (size_t)(p->T + 1) * p->nlat * 4 * (p->prec == PFSH_FP64 ? 16 : 8);
  if (cudaMalloc(&p->F2, bytes) != cudaSuccess) {
    cudaGetLastError();
    p->F2 = nullptr;
    return fail(PFSH_ENOMEM, "chain_prepare: second Fourier buffer");
  }
  p->device_bytes += bytes;
  return PFSH_OK;
}

// Step C for slices n0..n1-1 of node-major arrays (node stride node_stride,
// slice stride slice_stride, in doubles): slice n receives the last node of
// slice n-1 (theta, F_E, F_I; for n = n0 only if recv_first) and performs one
// sweep with its FAS term.  The level must hold one state (B = 1).
// `after_first` (optional) is recorded after the first launch, which holds
// the receive of slice n0: from then on slice n0-1 may be overwritten.
int chain_sweeps(sdc_level *l, double *th, double *fe, double *fi, const double *tau, size_t node_stride,
                 size_t slice_stride, int n0, int n1, bool recv_first, cudaStream_t s, cudaEvent_t after_first) {
  const sht_plan *p = l->ctx->plan;
  if (l->nodes - 1 > 8) return fail(PFSH_EUNSUPPORTED, "chain_sweeps: more than 9 nodes");
  if (coriolis_implicit(l->ctx->prm) && !l->d_band) return fail(PFSH_EINVAL, "chain_sweeps: no banded factors");
  if (p->prec == PFSH_FP64)
    return chain_typed<double>(l, chain_geo<double>(l->ctx, p->d_P, SpecTables<double>{p->d_eps, p->d_ilap}), th,
                               fe, fi, tau, node_stride, slice_stride, n0, n1, recv_first, s, after_first);
  return chain_typed<float>(l, chain_geo<float>(l->ctx, p->d_P32, SpecTables<float>{p->d_eps32, p->d_ilap32}), th,
                            fe, fi, tau, node_stride, slice_stride, n0, n1, recv_first, s, after_first);
}

}  // namespace pfsh
