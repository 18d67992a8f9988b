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
      if ((rc = chain_node_launch<R>(st, g, c, s, n > n0 || k > 1))) return rc;
      if (after_first && n == n0 && k == 1) PFSH_CUDA(cudaEventRecord(after_first, s));
      if ((rc = grid_rhs(p, 1, ctx->prm, s, true))) return rc;
    }
  }
  if (n1 > n0) {   // analysis of the last slice's last node
    ChainStep st = {};
    st.a_th = TH + (n1 - 1) * ss + M * ns;
    st.a_fe = FE + (n1 - 1) * ss + M * ns;
    st.a_fi = FI + (n1 - 1) * ss + M * ns;
    if ((rc = chain_node_launch<R>(st, g, c, s, true))) return rc;
  }
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
