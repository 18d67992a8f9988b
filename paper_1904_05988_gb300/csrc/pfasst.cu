// Two-level PFASST over n_ts time slices held on one GPU (Sections 5.1.2,
// 5.2, 5.3 and Algorithm 1).
//
// The paper's processors P_n become slice indices of node-major arrays
// [node][slice][3][ncoef]; a "send" to the next processor is a device copy.
// Step A (fine sweep) and Step B (restriction, coarse F, FAS) run batched
// over a group of consecutive slices; Step C (coarse sweeps) is a chain in
// slice order; Step D (interpolation of increments, new initial values,
// node-0 F) is batched over a group again.
//
// Within one iteration Step C of group g depends only on Steps A/B of group
// g and on Step C of group g-1, so the chain runs on a second stream and
// overlaps Steps A/B of the later groups; Step D of group g waits for Step C
// of group g.  The arithmetic of every slice is the same for any grouping
// as long as each group holds at least kMinGroupSlices slices (the RHS path
// for batches of one or two states differs from the batched one).
#include <math.h>

#include <stdlib.h>

#include <algorithm>
#include <new>

#include "internal.cuh"

namespace pfsh {

constexpr int kMinGroupSlices = 4;

struct Mat16 {
  double v[16][16];
};

__device__ __forceinline__ int tri_m2(int idx, int T) {
  const float b = 2.f * T + 3.f;
  int m = (int)((b - sqrtf(fmaxf(b * b - 8.f * idx, 0.f))) * 0.5f);
  m = max(0, min(m, T));
  while (m > 0 && poff(T, m) > idx) --m;
  while (m < T && poff(T, m + 1) <= idx) ++m;
  return m;
}

// tau_c[i] = dt D( sum_k Rt[i][k] sum_j Qf[k][j] F_f,j ) - dt sum_j Qc[i][j] F_c,j
// (FAS correction of Eq. tau_term_level_l+1 with tau_f = 0; the Theta terms
// of A_c(R Theta_f) - R A_f(Theta_f) cancel.)  MF, MC bound the node counts
// at compile time (nf <= MF, ncn <= MC) so that the per-node values stay in
// registers.  The same pass saves theta_c, F_E,c and F_I,c of every coarse
// node (th_cs, fe_cs, fi_cs: the values Step D takes the coarse increment
// against), since it reads the two right-hand sides anyway.
template <int MF, int MC>
__global__ void k_fas(int Tf, int Tc, int nts, int nf, int ncn, double dt, Mat16 RQf, Mat16 Qc,
                      const double2 *__restrict__ fe_f, const double2 *__restrict__ fi_f,
                      const double2 *__restrict__ fe_c, const double2 *__restrict__ fi_c,
                      double2 *__restrict__ tau, const double2 *__restrict__ th_c, double2 *__restrict__ th_cs,
                      double2 *__restrict__ fe_cs, double2 *__restrict__ fi_cs) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  const int ncc = ncoef_of(Tc), ncf = ncoef_of(Tf);
  if (idx >= ncc) return;
  const int m = tri_m2(idx, Tc);
  const int fidx = poff(Tf, m) + (idx - poff(Tc, m));
  const size_t fs = (size_t)nts * 3 * ncf, cs = (size_t)nts * 3 * ncc;
  {
    const int f = blockIdx.z;   // one field per grid layer
    const size_t fo = (size_t)b * 3 * ncf + (size_t)f * ncf + fidx;
    const size_t co = (size_t)b * 3 * ncc + (size_t)f * ncc + idx;
    double2 Ff[MF], Fc[MC];
#pragma unroll
    for (int k = 0; k < MF; ++k)
      if (k < nf) Ff[k] = fe_f[k * fs + fo] + fi_f[k * fs + fo];
#pragma unroll
    for (int k = 0; k < MC; ++k)
      if (k < ncn) {
        const double2 e = fe_c[k * cs + co], g = fi_c[k * cs + co];
        Fc[k] = e + g;
        fe_cs[k * cs + co] = e;
        fi_cs[k * cs + co] = g;
        th_cs[k * cs + co] = th_c[k * cs + co];
      }
#pragma unroll
    for (int i = 0; i < MC; ++i) {
      if (i >= ncn) break;
      double2 a = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < MF; ++k)
        if (k < nf) {
          a.x += RQf.v[i][k] * Ff[k].x;
          a.y += RQf.v[i][k] * Ff[k].y;
        }
      double2 c = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < MC; ++k)
        if (k < ncn) {
          c.x += Qc.v[i][k] * Fc[k].x;
          c.y += Qc.v[i][k] * Fc[k].y;
        }
      tau[i * cs + co] = make_double2(dt * a.x - dt * c.x, dt * a.y - dt * c.y);
    }
  }
}

// x_f[k] += sum_i Pt[k][i] Z(x_c[i] - x_cs[i]) for fine nodes k >= kmin and
// the coefficients the coarse level holds (zero-padding elsewhere); node
// counts bounded at compile time as in k_fas.
// The three arrays (theta, F_E, F_I) in one launch: grid layer z = 3 q + f
// takes field f of array q.
struct InterpArrays {
  const double2 *xc[3], *xcs[3];
  double2 *xf[3];
};

template <int MF, int MC>
__global__ void k_interp_inc(int Tf, int Tc, int nts, int nf, int ncn, int kmin, Mat16 Pt, InterpArrays arr) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  const int q = blockIdx.z / 3;
  const double2 *__restrict__ xc = arr.xc[q];
  const double2 *__restrict__ xcs = arr.xcs[q];
  double2 *__restrict__ xf = arr.xf[q];
  const int ncc = ncoef_of(Tc), ncf = ncoef_of(Tf);
  if (idx >= ncc) return;
  const int m = tri_m2(idx, Tc);
  const int fidx = poff(Tf, m) + (idx - poff(Tc, m));
  const size_t fs = (size_t)nts * 3 * ncf, cs = (size_t)nts * 3 * ncc;
  {
    const int f = blockIdx.z - 3 * q;   // field f of array q
    const size_t fo = (size_t)b * 3 * ncf + (size_t)f * ncf + fidx;
    const size_t co = (size_t)b * 3 * ncc + (size_t)f * ncc + idx;
    double2 d[MC];
#pragma unroll
    for (int i = 0; i < MC; ++i)
      if (i < ncn) d[i] = xc[i * cs + co] - xcs[i * cs + co];
#pragma unroll
    for (int k = 0; k < MF; ++k) {
      if (k >= nf) break;
      if (k < kmin) continue;
      double2 a = make_double2(0.0, 0.0);
#pragma unroll
      for (int i = 0; i < MC; ++i)
        if (i < ncn) {
          a.x += Pt.v[k][i] * d[i].x;
          a.y += Pt.v[k][i] * d[i].y;
        }
      double2 v = xf[k * fs + fo];
      xf[k * fs + fo] = v + a;
    }
  }
}

// Residual check: per slice b, max |theta_f(end) - prev| / max |theta_f(end)|
// over the slice's coefficients (one block per slice), then prev = current.
__global__ void k_residual(size_t n2, const double2 *__restrict__ cur, double2 *__restrict__ prev,
                           double *__restrict__ res) {
  __shared__ double sd[32], sv[32];
  const int b = blockIdx.x;
  const double2 *c = cur + (size_t)b * n2;
  double2 *p = prev + (size_t)b * n2;
  double md = 0.0, mv = 0.0;
  for (size_t e = threadIdx.x; e < n2; e += blockDim.x) {
    const double2 x = c[e], y = p[e];
    md = fmax(md, fmax(fabs(x.x - y.x), fabs(x.y - y.y)));
    mv = fmax(mv, fmax(fabs(x.x), fabs(x.y)));
    p[e] = x;
  }
  for (int d = 16; d > 0; d >>= 1) {
    md = fmax(md, __shfl_xor_sync(0xffffffffu, md, d));
    mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, d));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
    sd[w] = md;
    sv[w] = mv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < nw; ++i) {
      md = fmax(md, sd[i]);
      mv = fmax(mv, sv[i]);
    }
    res[b] = mv > 0.0 ? md / mv : md;
  }
}

// Three device copies of the same shape in one launch: rows x n2 complex
// elements, row pitches spitch / dpitch (complex elements); layer z = array.
struct Copy3 {
  const double2 *src[3];
  double2 *dst[3];
};

__global__ void k_copy3(Copy3 c, size_t n2, size_t spitch, size_t dpitch) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y, q = blockIdx.z;
  if (e < n2) c.dst[q][(size_t)row * dpitch + e] = c.src[q][(size_t)row * spitch + e];
}

static int copy3(const double *const src[3], double *const dst[3], size_t n2, int rows, size_t spitch,
                 size_t dpitch, cudaStream_t s) {
  Copy3 c;
  for (int q = 0; q < 3; ++q) {
    c.src[q] = (const double2 *)src[q];
    c.dst[q] = (double2 *)dst[q];
  }
  {
    PFSH_LAUNCH("k_copy3", s);
    k_copy3<<<dim3((unsigned)((n2 + 255) / 256), rows, 3), 256, 0, s>>>(c, n2, spitch, dpitch);
  }
  PFSH_CHECK_LAUNCH("k_copy3");
  return PFSH_OK;
}

// Predictor start: the restricted initial value (state 0 of base_c) and its
// right-hand sides (state 0 of fe_c, fi_c) copied to every slice of base_c
// and to every (node, slice) of th_c, fe_c, fi_c; grid.y = (node, slice).
__global__ void k_broadcast(size_t n2, int nts, const double2 *__restrict__ base, const double2 *__restrict__ fe0,
                            const double2 *__restrict__ fi0, double2 *__restrict__ th, double2 *fe, double2 *fi,
                            double2 *base_all) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int ns = blockIdx.y, slice = ns % nts;
  if (e >= n2) return;
  const double2 b = base[e], ve = fe0[e], vi = fi0[e];   // state 0 is only read
  th[(size_t)ns * n2 + e] = b;
  if (ns > 0) {
    fe[(size_t)ns * n2 + e] = ve;
    fi[(size_t)ns * n2 + e] = vi;
  }
  if (ns < nts && slice > 0) base_all[(size_t)slice * n2 + e] = b;
}

// Predictor: x_f[k][b] = theta0 + sum_i Pt[k][i] Z(x_c[i][b] - base_c[b])
template <int MF, int MC>
__global__ void k_pred_interp(int Tf, int Tc, int nts, int nf, int ncn, Mat16 Pt, const double2 *__restrict__ th0,
                              const double2 *__restrict__ xc, const double2 *__restrict__ basec,
                              double2 *__restrict__ xf) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  const int ncc = ncoef_of(Tc), ncf = ncoef_of(Tf);
  if (idx >= ncf) return;
  const int m = tri_m2(idx, Tf);
  const int n = m + (idx - poff(Tf, m));
  const size_t fs = (size_t)nts * 3 * ncf, cs = (size_t)nts * 3 * ncc;
  const bool low = (n <= Tc);
  const int cidx = low ? poff(Tc, m) + (n - m) : 0;
  {
    const int f = blockIdx.z;   // one field per grid layer
    const double2 base = th0[(size_t)f * ncf + idx];
    double2 d[MC];
    if (low) {
      const size_t co = (size_t)b * 3 * ncc + (size_t)f * ncc + cidx;
      const double2 bc = basec[(size_t)b * 3 * ncc + (size_t)f * ncc + cidx];
#pragma unroll
      for (int i = 0; i < MC; ++i)
        if (i < ncn) d[i] = xc[i * cs + co] - bc;
    }
#pragma unroll
    for (int k = 0; k < MF; ++k) {
      if (k >= nf) break;
      double2 v = base;
      if (low) {
        double2 a = make_double2(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < MC; ++i)
          if (i < ncn) {
            a.x += Pt.v[k][i] * d[i].x;
            a.y += Pt.v[k][i] * d[i].y;
          }
        v = v + a;
      }
      xf[k * fs + (size_t)b * 3 * ncf + (size_t)f * ncf + idx] = v;
    }
  }
}

// Step D, last line of Algorithm 1: theta_f^{n,0} = sent^{n-1} +
// Z(theta_c^{n,0} - D sent^{n-1}) for slices n >= 1; slice b = first +
// blockIdx.y relative to the base pointers (sent[b-1] must exist).
__global__ void k_node0(int Tf, int Tc, int first, const double2 *__restrict__ sent,
                        const double2 *__restrict__ thc0, double2 *__restrict__ thf0) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y + first;
  const int ncc = ncoef_of(Tc), ncf = ncoef_of(Tf);
  if (idx >= ncf) return;
  const int m = tri_m2(idx, Tf);
  const int n = m + (idx - poff(Tf, m));
  {
    const int f = blockIdx.z;   // one field per grid layer
    double2 v = sent[(size_t)(b - 1) * 3 * ncf + (size_t)f * ncf + idx];
    if (n <= Tc) {
      const double2 c = thc0[(size_t)b * 3 * ncc + (size_t)f * ncc + poff(Tc, m) + (n - m)];
      v = v + (c - v);
    }
    thf0[(size_t)b * 3 * ncf + (size_t)f * ncf + idx] = v;
  }
}

}  // namespace pfsh

using namespace pfsh;

static void pf_free(pfasst *pf) {
  if (!pf) return;
  double *bufs[] = {pf->th_f, pf->fe_f, pf->fi_f, pf->th_c, pf->fe_c, pf->fi_c, pf->th_cs,
                    pf->fe_cs, pf->fi_cs, pf->tau, pf->sent, pf->base_c, pf->theta0, pf->prev_end};
  for (double *b : bufs)
    if (b) cudaFree(b);
  for (auto &e : pf->graphs_.e)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  if (pf->cap_stream) cudaStreamDestroy(pf->cap_stream);
  if (pf->chain_stream) cudaStreamDestroy(pf->chain_stream);
  if (pf->ev_fork) cudaEventDestroy(pf->ev_fork);
  for (int g = 0; g < pfasst::kMaxGroups; ++g) {
    if (pf->ev_B[g]) cudaEventDestroy(pf->ev_B[g]);
    if (pf->ev_C[g]) cudaEventDestroy(pf->ev_C[g]);
    if (pf->ev_R[g]) cudaEventDestroy(pf->ev_R[g]);
  }
  sdc_level_destroy(pf->lev_cc);
  swe_ctx_destroy(pf->ctx_cc);
  sht_plan_destroy(pf->plan_cc);
  sdc_level_destroy(pf->lev_f);
  sdc_level_destroy(pf->lev_c);
  swe_ctx_destroy(pf->ctx_f);
  swe_ctx_destroy(pf->ctx_c);
  sht_plan_destroy(pf->plan_f);
  sht_plan_destroy(pf->plan_c);
  delete pf;
}

extern "C" int pfasst_create(pfasst **out, const pfasst_config *cfg) {
  if (!out || !cfg) return fail(PFSH_EINVAL, "pfasst_create: NULL argument");
  *out = nullptr;
  const pfasst_config &c = *cfg;
  if (c.n_ts < 1 || c.fine_nodes < 2 || c.fine_nodes > 9 || c.coarse_nodes < 2 || c.coarse_nodes > 9)
    return fail(PFSH_EINVAL, "pfasst_create: need n_ts >= 1 and 2..9 nodes per level");
  if (c.Tc > c.Tf || c.Tc < 1) return fail(PFSH_EINVAL, "pfasst_create: need 1 <= Tc <= Tf");
  if (c.slice_groups < 0) return fail(PFSH_EINVAL, "pfasst_create: slice_groups must be >= 0");
  if (!(c.dt > 0)) return fail(PFSH_EINVAL, "pfasst_create: dt must be > 0");
  pfasst *pf = new (std::nothrow) pfasst();
  if (!pf) return fail(PFSH_ENOMEM, "pfasst_create");
  pf->cfg = c;
  pf->Mf = c.fine_nodes - 1;
  pf->Mc = c.coarse_nodes - 1;
  const int nts = c.n_ts;
  // fine passes: sweep batches of n_ts states; coarse: (Mc+1) n_ts states in Step B
  int mb_f = 5 * std::min(nts, 32);
  int mb_c = 5 * std::min(nts * c.coarse_nodes, 96);
  int rc;
  if ((rc = sht_plan_create(&pf->plan_f, c.Tf, c.nlat_f, c.nlon_f, mb_f, c.prec)) ||
      (rc = sht_plan_create(&pf->plan_c, c.Tc, c.nlat_c, c.nlon_c, mb_c, c.prec)) ||
      (rc = swe_ctx_create(&pf->ctx_f, pf->plan_f, &c.phys)) ||
      (rc = swe_ctx_create(&pf->ctx_c, pf->plan_c, &c.phys)) ||
      (rc = sdc_level_create(&pf->lev_f, pf->ctx_f, c.fine_nodes, c.dt, nts)) ||
      (rc = sdc_level_create(&pf->lev_c, pf->ctx_c, c.coarse_nodes, c.dt, nts)) ||
      (rc = sht_plan_create(&pf->plan_cc, c.Tc, c.nlat_c, c.nlon_c, 5, c.prec)) ||
      (rc = swe_ctx_create(&pf->ctx_cc, pf->plan_cc, &c.phys)) ||
      (rc = sdc_level_create(&pf->lev_cc, pf->ctx_cc, c.coarse_nodes, c.dt, 1))) {
    pf_free(pf);
    return rc;
  }
  pf->sf = (size_t)3 * ncoef_of(c.Tf) * 2;
  pf->sc = (size_t)3 * ncoef_of(c.Tc) * 2;
  struct A {
    double **p;
    size_t n;
  } allocs[] = {{&pf->th_f, (size_t)(pf->Mf + 1) * nts * pf->sf}, {&pf->fe_f, (size_t)(pf->Mf + 1) * nts * pf->sf},
                {&pf->fi_f, (size_t)(pf->Mf + 1) * nts * pf->sf}, {&pf->th_c, (size_t)(pf->Mc + 1) * nts * pf->sc},
                {&pf->fe_c, (size_t)(pf->Mc + 1) * nts * pf->sc}, {&pf->fi_c, (size_t)(pf->Mc + 1) * nts * pf->sc},
                {&pf->th_cs, (size_t)(pf->Mc + 1) * nts * pf->sc}, {&pf->fe_cs, (size_t)(pf->Mc + 1) * nts * pf->sc},
                {&pf->fi_cs, (size_t)(pf->Mc + 1) * nts * pf->sc}, {&pf->tau, (size_t)(pf->Mc + 1) * nts * pf->sc},
                {&pf->sent, (size_t)2 * nts * pf->sf},            {&pf->base_c, (size_t)nts * pf->sc},
                {&pf->theta0, pf->sf},                            {&pf->prev_end, (size_t)nts * pf->sf}};
  for (auto &a : allocs) {
    if (cudaMalloc(a.p, a.n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      pf_free(pf);
      return fail(PFSH_ENOMEM, "pfasst_create: device arrays");
    }
    cudaMemset(*a.p, 0, a.n * sizeof(double));
  }
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  bool ok = cudaStreamCreateWithFlags(&pf->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithPriority(&pf->chain_stream, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
            cudaEventCreateWithFlags(&pf->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int g = 0; ok && g < pfasst::kMaxGroups; ++g)
    ok = cudaEventCreateWithFlags(&pf->ev_B[g], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&pf->ev_C[g], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&pf->ev_R[g], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pf_free(pf);
    return fail(PFSH_ECUDA, "pfasst_create: streams/events");
  }
  {
    const char *e = getenv("PFSH_NO_GRAPH");
    pf->graphs = !(e && e[0] && e[0] != '0');
    // slice groups, each of >= kMinGroupSlices slices; by default 2 for the
    // mixed forms (their fine sweeps leave room for the chain), 1 for FP64
    // (its FP64-bound fine sweeps lose more from smaller batches than the
    // overlap gains)
    const int g = c.slice_groups > 0 ? c.slice_groups : (c.prec == PFSH_FP64 ? 1 : 2);
    pf->groups = std::max(1, std::min(g, std::min(pfasst::kMaxGroups, nts / kMinGroupSlices)));
  }
  lagrange_matrix(pf->lev_f->tau_nodes, c.fine_nodes, pf->lev_c->tau_nodes, c.coarse_nodes, pf->Rt);
  lagrange_matrix(pf->lev_c->tau_nodes, c.coarse_nodes, pf->lev_f->tau_nodes, c.fine_nodes, pf->Pt);
  *out = pf;
  return PFSH_OK;
}

extern "C" int pfasst_destroy(pfasst *pf) {
  if (!pf) return PFSH_OK;
  cudaDeviceSynchronize();
  pf_free(pf);
  return PFSH_OK;
}

extern "C" int pfasst_set_initial(pfasst *pf, const double *theta0, pfsh_stream_t stream) {
  if (!pf || !theta0) return fail(PFSH_EINVAL, "pfasst_set_initial: NULL argument");
  PFSH_CUDA(cudaMemcpyAsync(pf->theta0, theta0, pf->sf * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return PFSH_OK;
}

// Predictor (Section 5.2.1): the restricted initial value is broadcast to
// every slice and node, then in round j the slices n >= j take slice n-1's
// round-(j-1) end value and sweep once on the coarse level (slice n sweeps
// n+1 times in all); the received value's right-hand sides are those the
// sender evaluated at its last node (the same state through the same
// kernels), so they travel with it.  Finally the coarse increments are
// interpolated to the fine nodes and the fine right-hand sides evaluated.
static int predict_body(pfasst *pf, cudaStream_t s) {
  const int nts = pf->cfg.n_ts, Mc = pf->Mc, Mf = pf->Mf;
  const size_t sc = pf->sc, sf = pf->sf;
  const size_t cnode = (size_t)nts * sc;
  int rc;
  // restricted initial value and its right-hand sides, broadcast
  double R1[16 * 16] = {0};
  R1[0] = 1.0;
  if ((rc = restrict_launch(R1, 1, 1, pf->theta0, sf, pf->base_c, sc, pf->cfg.Tf, pf->cfg.Tc, 1, s))) return rc;
  if ((rc = rhs_eval(pf->ctx_c, pf->base_c, pf->fe_c, pf->fi_c, 1, s))) return rc;
  {
    const size_t n2 = sc / 2;   // complex elements per state
    PFSH_LAUNCH("k_broadcast", s);
    dim3 g((unsigned)((n2 + 255) / 256), (unsigned)(Mc + 1) * nts);
    k_broadcast<<<g, 256, 0, s>>>(n2, nts, (const double2 *)pf->base_c, (const double2 *)pf->fe_c,
                                  (const double2 *)pf->fi_c, (double2 *)pf->th_c, (double2 *)pf->fe_c,
                                  (double2 *)pf->fi_c, (double2 *)pf->base_c);
  }
  PFSH_CHECK_LAUNCH("k_broadcast");
  // rounds: slices n >= j take slice n-1's round j-1 end value and sweep
  for (int j = 0; j < nts; ++j) {
    const int cnt = nts - j;
    if (j > 0) {   // node 0 of slices j.. <- last node of slices j-1.. (distinct nodes: no overlap)
      const size_t from = Mc * cnode + (j - 1) * sc, to = j * sc;
      const double *src[3] = {pf->th_c + from, pf->fe_c + from, pf->fi_c + from};
      double *const dst[3] = {pf->th_c + to, pf->fe_c + to, pf->fi_c + to};
      if ((rc = copy3(src, dst, cnt * sc / 2, 1, 0, 0, s))) return rc;
    }
    if ((rc = sdc_sweep_strided(pf->lev_c, pf->th_c + j * sc, pf->fe_c + j * sc, pf->fi_c + j * sc, nullptr, cnode,
                                cnt, s)))
      return rc;
  }
  // fine prediction: theta0 + interpolated coarse increment, then fine F everywhere
  Mat16 P;
  for (int i = 0; i < 16; ++i)
    for (int k = 0; k < 16; ++k) P.v[i][k] = pf->Pt[i][k];
  dim3 g((ncoef_of(pf->cfg.Tf) + 255) / 256, nts, 3);
  {
    PFSH_LAUNCH("k_pred_interp", s);
    auto kern = (Mf + 1 == 5 && Mc + 1 == 3) ? k_pred_interp<5, 3> : k_pred_interp<9, 9>;
    kern<<<g, 256, 0, s>>>(pf->cfg.Tf, pf->cfg.Tc, nts, Mf + 1, Mc + 1, P, (const double2 *)pf->theta0,
                                    (const double2 *)pf->th_c, (const double2 *)pf->base_c, (double2 *)pf->th_f);
  }
  PFSH_CHECK_LAUNCH("k_pred_interp");
  return rhs_eval(pf->ctx_f, pf->th_f, pf->fe_f, pf->fi_f, (Mf + 1) * nts, s);
}

// Steps A and B for slices [g0, g0 + cnt): fine sweep, send, restriction,
// coarse F at every node, saved copies, FAS correction.
static int steps_AB(pfasst *pf, int g0, int cnt, int par, cudaStream_t s) {
  const pfasst_config &c = pf->cfg;
  const int nts = c.n_ts, Mc = pf->Mc, Mf = pf->Mf;
  const size_t sc = pf->sc, sf = pf->sf;
  const size_t cnode = (size_t)nts * sc, fnode = (size_t)nts * sf;
  int rc;
  if ((rc = sdc_sweep_strided(pf->lev_f, pf->th_f + g0 * sf, pf->fe_f + g0 * sf, pf->fi_f + g0 * sf, nullptr, fnode,
                              cnt, s)))
    return rc;
  PFSH_CUDA(cudaMemcpyAsync(pf->sent + (par * nts + g0) * sf, pf->th_f + Mf * fnode + g0 * sf, cnt * sf * 8,
                            cudaMemcpyDeviceToDevice, s));
  {
    double R[16 * 16];
    for (int i = 0; i < 16; ++i)
      for (int k = 0; k < 16; ++k) R[i * 16 + k] = pf->Rt[i][k];
    if ((rc = restrict_launch(R, Mf + 1, Mc + 1, pf->th_f + g0 * sf, fnode, pf->th_c + g0 * sc, cnode, c.Tf, c.Tc,
                              cnt, s)))
      return rc;
  }
  // coarse F at every node: one pass over the (Mc+1) x cnt states
  if ((rc = rhs_eval_nodes(pf->ctx_c, pf->th_c + g0 * sc, pf->fe_c + g0 * sc, pf->fi_c + g0 * sc, Mc + 1, cnt, cnode,
                           s)))
    return rc;
  // (the saved coarse copies for Step D are written by k_fas below)
  Mat16 RQf, Qc;
  for (int i = 0; i < 16; ++i)
    for (int k = 0; k < 16; ++k) {
      RQf.v[i][k] = 0.0;
      Qc.v[i][k] = 0.0;
    }
  for (int i = 0; i <= Mc; ++i) {
    for (int k = 0; k <= Mf; ++k) {
      double acc = 0.0;
      for (int q = 0; q <= Mf; ++q) acc += pf->Rt[i][q] * pf->lev_f->Q[q][k];
      RQf.v[i][k] = acc;
    }
    for (int k = 0; k <= Mc; ++k) Qc.v[i][k] = pf->lev_c->Q[i][k];
  }
  dim3 g((ncoef_of(c.Tc) + 255) / 256, cnt, 3);
  {
    PFSH_LAUNCH("k_fas", s);
    auto kern = (Mf + 1 == 5 && Mc + 1 == 3) ? k_fas<5, 3> : k_fas<9, 9>;
    kern<<<g, 256, 0, s>>>(c.Tf, c.Tc, nts, Mf + 1, Mc + 1, c.dt, RQf, Qc, (const double2 *)(pf->fe_f + g0 * sf),
                            (const double2 *)(pf->fi_f + g0 * sf), (const double2 *)(pf->fe_c + g0 * sc),
                            (const double2 *)(pf->fi_c + g0 * sc), (double2 *)(pf->tau + g0 * sc),
                            (const double2 *)(pf->th_c + g0 * sc), (double2 *)(pf->th_cs + g0 * sc),
                            (double2 *)(pf->fe_cs + g0 * sc), (double2 *)(pf->fi_cs + g0 * sc));
  }
  PFSH_CHECK_LAUNCH("k_fas");
  return PFSH_OK;
}

// Step C for slices [g0, g0 + cnt) in slice order: receive slice n-1's coarse
// end value (with its right-hand sides), one coarse sweep with the FAS term.
static int step_C(pfasst *pf, int g0, int cnt, cudaStream_t s, cudaEvent_t received) {
  const size_t sc = pf->sc, cnode = (size_t)pf->cfg.n_ts * sc;
  return chain_sweeps(pf->lev_cc, pf->th_c, pf->fe_c, pf->fi_c, pf->tau, cnode, sc, g0, g0 + cnt, g0 > 0, s,
                      received);
}

// Step D for slices [g0, g0 + cnt): interpolate the coarse increments into
// fine nodes >= 1, new fine initial values (slices >= 1), fine node-0 F.
static int step_D(pfasst *pf, int g0, int cnt, int par, cudaStream_t s) {
  const pfasst_config &c = pf->cfg;
  const int nts = c.n_ts, Mc = pf->Mc, Mf = pf->Mf;
  const size_t sc = pf->sc, sf = pf->sf;
  Mat16 P;
  for (int i = 0; i < 16; ++i)
    for (int k = 0; k < 16; ++k) P.v[i][k] = pf->Pt[i][k];
  dim3 g((ncoef_of(c.Tc) + 255) / 256, cnt, 9);
  const double *xc[3] = {pf->th_c, pf->fe_c, pf->fi_c};
  const double *xs[3] = {pf->th_cs, pf->fe_cs, pf->fi_cs};
  double *xf[3] = {pf->th_f, pf->fe_f, pf->fi_f};
  InterpArrays arr;
  for (int q = 0; q < 3; ++q) {
    arr.xc[q] = (const double2 *)(xc[q] + g0 * sc);
    arr.xcs[q] = (const double2 *)(xs[q] + g0 * sc);
    arr.xf[q] = (double2 *)(xf[q] + g0 * sf);
  }
  {
    PFSH_LAUNCH("k_interp_inc", s);
    auto kern = (Mf + 1 == 5 && Mc + 1 == 3) ? k_interp_inc<5, 3> : k_interp_inc<9, 9>;
    kern<<<g, 256, 0, s>>>(c.Tf, c.Tc, nts, Mf + 1, Mc + 1, 1, P, arr);
  }
  PFSH_CHECK_LAUNCH("k_interp_inc");
  const int first = g0 == 0 ? 1 : 0;
  if (cnt - first > 0) {
    dim3 g0d((ncoef_of(c.Tf) + 255) / 256, cnt - first, 3);
    {
      PFSH_LAUNCH("k_node0", s);
      k_node0<<<g0d, 256, 0, s>>>(c.Tf, c.Tc, first, (const double2 *)(pf->sent + ((size_t)par * nts + g0) * sf),
                                  (const double2 *)(pf->th_c + g0 * sc), (double2 *)(pf->th_f + g0 * sf));
    }
    PFSH_CHECK_LAUNCH("k_node0");
  }
  return rhs_eval(pf->ctx_f, pf->th_f + g0 * sf, pf->fe_f + g0 * sf, pf->fi_f + g0 * sf, cnt, s);
}

// `count` iterations of Algorithm 1, the last of them Step A only when
// `last`.  Steps A/B of slice group g run on `s`, Step C of every group on
// the chain stream, Step D of group g on `s` again.  Across iterations the
// groups form a wavefront: Steps D/A/B of group g in iteration k+1 wait only
// for Step C of group g in iteration k (and Step B of group g also for the
// receive of group g+1 in iteration k, whose first launch reads group g's
// last slice), so the fine sweeps of the early groups of iteration k+1 run
// beside the coarse chain of the late groups of iteration k.  The values
// sent in Step A are double-buffered by iteration parity because Step D of
// group g+1 in iteration k reads them after Step A of group g in iteration
// k+1 has run.
static int block_body(pfasst *pf, int count, int last, cudaStream_t s) {
  const int nts = pf->cfg.n_ts;
  const int nfull = count - (last ? 1 : 0);
  const int G = pf->groups;
  auto group = [&](int g, int *g0, int *cnt) {
    *g0 = (int)((long)nts * g / G);
    *cnt = (int)((long)nts * (g + 1) / G) - *g0;
  };
  // with the event profiler on, everything runs on `s` so that per-launch
  // durations are not stretched by the overlap
  cudaStream_t cs = profiler_on() ? s : pf->chain_stream;
  int rc, g0, cnt;
  if (nfull > 0) {
    PFSH_CUDA(cudaEventRecord(pf->ev_fork, s));
    PFSH_CUDA(cudaStreamWaitEvent(cs, pf->ev_fork, 0));
  }
  for (int it = 0; it < nfull; ++it) {
    for (int g = 0; g < G; ++g) {
      group(g, &g0, &cnt);
      if (it > 0) {
        PFSH_CUDA(cudaStreamWaitEvent(s, pf->ev_C[g], 0));
        if ((rc = step_D(pf, g0, cnt, (it - 1) & 1, s))) return rc;
        if (g + 1 < G) PFSH_CUDA(cudaStreamWaitEvent(s, pf->ev_R[g + 1], 0));
      }
      if ((rc = steps_AB(pf, g0, cnt, it & 1, s))) return rc;
      PFSH_CUDA(cudaEventRecord(pf->ev_B[g], s));
      PFSH_CUDA(cudaStreamWaitEvent(cs, pf->ev_B[g], 0));
      if ((rc = step_C(pf, g0, cnt, cs, g > 0 ? pf->ev_R[g] : nullptr))) return rc;
      PFSH_CUDA(cudaEventRecord(pf->ev_C[g], cs));
    }
  }
  for (int g = 0; nfull > 0 && g < G; ++g) {
    group(g, &g0, &cnt);
    PFSH_CUDA(cudaStreamWaitEvent(s, pf->ev_C[g], 0));
    if ((rc = step_D(pf, g0, cnt, (nfull - 1) & 1, s))) return rc;
  }
  if (last)   // the last iteration ends after the fine sweep (Step A)
    return sdc_sweep_strided(pf->lev_f, pf->th_f, pf->fe_f, pf->fi_f, nullptr, (size_t)nts * pf->sf, nts, s);
  return PFSH_OK;
}

// A block of iterations is a fixed sequence of launches on fixed buffers
// over several streams, so it is recorded once into a CUDA graph (on a
// private capture stream that the other streams join) per (count, last) and
// replayed on the caller's stream; the first call of each key runs eagerly,
// which also sets every kernel attribute before capture.  Profiling or
// PFSH_NO_GRAPH=1 keeps the eager path.
template <typename Body>
static int run_cached(GraphCache &cache, bool graphs, cudaStream_t cap, int count, int last, cudaStream_t s,
                      Body body) {
  if (!graphs || profiler_on()) return body(s);
  GraphEntry *e = nullptr;
  for (auto &x : cache.e)
    if (x.calls > 0 && x.count == count && x.last == last) e = &x;
  if (!e) {
    for (auto &x : cache.e)
      if (x.calls == 0) {
        e = &x;
        break;
      }
    if (!e) return body(s);   // cache full: eager
    e->count = count;
    e->last = last;
  }
  if (e->exec) {
    PFSH_CUDA(cudaGraphLaunch(e->exec, s));
    count_launches(e->launches);
    return PFSH_OK;
  }
  if (e->calls++ == 0) return body(s);
  cudaGraph_t g = nullptr;
  PFSH_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  const unsigned long long n0 = launches_so_far();
  int rc = body(cap);
  const unsigned long long n1 = launches_so_far();
  cudaError_t err = cudaStreamEndCapture(cap, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (err != cudaSuccess) return cuda_fail(err, "pfasst: cudaStreamEndCapture");
  err = cudaGraphInstantiateWithFlags(&e->exec, g, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(g);
  if (err != cudaSuccess) {
    e->exec = nullptr;
    return cuda_fail(err, "pfasst: cudaGraphInstantiate");
  }
  e->launches = n1 - n0;
  g_launches_uncount(n1 - n0);
  PFSH_CUDA(cudaGraphLaunch(e->exec, s));
  count_launches(e->launches);
  return PFSH_OK;
}

static int run_block(pfasst *pf, int count, int last, cudaStream_t s) {
  return run_cached(pf->graphs_, pf->graphs, pf->cap_stream, count, last, s,
                    [&](cudaStream_t st) { return block_body(pf, count, last, st); });
}

// opt-in non-finite check of the fine end values of every slice (outside the graphs)
static int check_ends(pfasst *pf, cudaStream_t s) {
  const size_t n = (size_t)pf->cfg.n_ts * pf->sf;
  return check_finite(pf->th_f + (size_t)pf->Mf * n, n, s);
}

extern "C" int pfasst_predict(pfasst *pf, pfsh_stream_t stream) {
  if (!pf) return fail(PFSH_EINVAL, "pfasst_predict: NULL argument");
  // graph key (0, 2): no iteration block has count 0
  int rc = run_cached(pf->graphs_, pf->graphs, pf->cap_stream, 0, 2, (cudaStream_t)stream,
                      [&](cudaStream_t st) { return predict_body(pf, st); });
  return rc ? rc : check_ends(pf, (cudaStream_t)stream);
}

extern "C" int pfasst_residual(pfasst *pf, double *res, pfsh_stream_t stream) {
  if (!pf || !res) return fail(PFSH_EINVAL, "pfasst_residual: NULL argument");
  const int nts = pf->cfg.n_ts;
  cudaStream_t s = (cudaStream_t)stream;
  {
    PFSH_LAUNCH("k_residual", s);
    k_residual<<<nts, 256, 0, s>>>(pf->sf / 2, (const double2 *)(pf->th_f + (size_t)pf->Mf * nts * pf->sf),
                                   (double2 *)pf->prev_end, res);
  }
  PFSH_CHECK_LAUNCH("k_residual");
  return PFSH_OK;
}

extern "C" int pfasst_iteration(pfasst *pf, int last, pfsh_stream_t stream) {
  if (!pf) return fail(PFSH_EINVAL, "pfasst_iteration: NULL argument");
  int rc = run_block(pf, 1, last ? 1 : 0, (cudaStream_t)stream);
  return rc ? rc : check_ends(pf, (cudaStream_t)stream);
}

extern "C" int pfasst_iterations(pfasst *pf, int count, int last, pfsh_stream_t stream) {
  if (!pf || count < 1) return fail(PFSH_EINVAL, "pfasst_iterations: NULL argument or count < 1");
  int rc = run_block(pf, count, last ? 1 : 0, (cudaStream_t)stream);
  return rc ? rc : check_ends(pf, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// ensembles of independent instances
// ---------------------------------------------------------------------------
static void ens_free(pfasst_ensemble *e) {
  if (!e) return;
  for (auto &x : e->graphs_.e)
    if (x.exec) cudaGraphExecDestroy(x.exec);
  for (int i = 0; i < e->n; ++i) {
    if (e->members && e->members[i]) pfasst_destroy(e->members[i]);
    if (e->streams && e->streams[i]) cudaStreamDestroy(e->streams[i]);
    if (e->ev_join && e->ev_join[i]) cudaEventDestroy(e->ev_join[i]);
  }
  if (e->ev_fork) cudaEventDestroy(e->ev_fork);
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  delete[] e->members;
  delete[] e->streams;
  delete[] e->ev_join;
  delete e;
}

extern "C" int pfasst_ensemble_create(pfasst_ensemble **out, const pfasst_config *cfgs, int n) {
  if (!out || !cfgs || n < 1) return fail(PFSH_EINVAL, "pfasst_ensemble_create: NULL argument or n < 1");
  *out = nullptr;
  pfasst_ensemble *e = new (std::nothrow) pfasst_ensemble();
  if (!e) return fail(PFSH_ENOMEM, "pfasst_ensemble_create");
  e->members = new (std::nothrow) pfasst *[n]();
  e->streams = new (std::nothrow) cudaStream_t[n]();
  e->ev_join = new (std::nothrow) cudaEvent_t[n]();
  if (!e->members || !e->streams || !e->ev_join) {
    ens_free(e);
    return fail(PFSH_ENOMEM, "pfasst_ensemble_create");
  }
  e->n = n;
  for (int i = 0; i < n; ++i) {
    int rc = pfasst_create(&e->members[i], &cfgs[i]);
    if (rc) {
      ens_free(e);
      return rc;
    }
    if (cudaStreamCreateWithFlags(&e->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_join[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ens_free(e);
      return fail(PFSH_ECUDA, "pfasst_ensemble_create: streams/events");
    }
  }
  if (cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ens_free(e);
    return fail(PFSH_ECUDA, "pfasst_ensemble_create: streams/events");
  }
  const char *env = getenv("PFSH_NO_GRAPH");
  e->graphs = !(env && env[0] && env[0] != '0');
  *out = e;
  return PFSH_OK;
}

extern "C" int pfasst_ensemble_destroy(pfasst_ensemble *e) {
  if (!e) return PFSH_OK;
  cudaDeviceSynchronize();
  ens_free(e);
  return PFSH_OK;
}

extern "C" pfasst *pfasst_ensemble_member(pfasst_ensemble *e, int i) {
  if (!e || i < 0 || i >= e->n) {
    fail(PFSH_EINVAL, "pfasst_ensemble_member: index out of range");
    return nullptr;
  }
  return e->members[i];
}

// fork every member onto its own stream, run `body(member, stream)`, join
template <typename Body>
static int ens_fanout(pfasst_ensemble *e, cudaStream_t s, Body body) {
  PFSH_CUDA(cudaEventRecord(e->ev_fork, s));
  for (int i = 0; i < e->n; ++i) {
    PFSH_CUDA(cudaStreamWaitEvent(e->streams[i], e->ev_fork, 0));
    int rc = body(e->members[i], e->streams[i]);
    if (rc) return rc;
    PFSH_CUDA(cudaEventRecord(e->ev_join[i], e->streams[i]));
    PFSH_CUDA(cudaStreamWaitEvent(s, e->ev_join[i], 0));
  }
  return PFSH_OK;
}

extern "C" int pfasst_ensemble_predict(pfasst_ensemble *e, pfsh_stream_t stream) {
  if (!e) return fail(PFSH_EINVAL, "pfasst_ensemble_predict: NULL argument");
  return ens_fanout(e, (cudaStream_t)stream,
                    [](pfasst *pf, cudaStream_t st) { return pfasst_predict(pf, (pfsh_stream_t)st); });
}

extern "C" int pfasst_ensemble_iterations(pfasst_ensemble *e, int count, int last, pfsh_stream_t stream) {
  if (!e || count < 1) return fail(PFSH_EINVAL, "pfasst_ensemble_iterations: NULL argument or count < 1");
  const int lst = last ? 1 : 0;
  return run_cached(e->graphs_, e->graphs, e->cap_stream, count, lst, (cudaStream_t)stream, [&](cudaStream_t st) {
    return ens_fanout(e, st, [&](pfasst *pf, cudaStream_t ms) { return block_body(pf, count, lst, ms); });
  });
}

extern "C" int pfasst_get(pfasst *pf, int level, int slice, int node, double *out, pfsh_stream_t stream) {
  if (!pf || !out) return fail(PFSH_EINVAL, "pfasst_get: NULL argument");
  const int nts = pf->cfg.n_ts;
  if (slice < 0 || slice >= nts) return fail(PFSH_EINVAL, "pfasst_get: slice out of range");
  const double *src;
  size_t st;
  if (level == 0) {
    if (node < 0 || node > pf->Mf) return fail(PFSH_EINVAL, "pfasst_get: node out of range");
    st = pf->sf;
    src = pf->th_f + ((size_t)node * nts + slice) * st;
  } else if (level == 1) {
    if (node < 0 || node > pf->Mc) return fail(PFSH_EINVAL, "pfasst_get: node out of range");
    st = pf->sc;
    src = pf->th_c + ((size_t)node * nts + slice) * st;
  } else {
    return fail(PFSH_EINVAL, "pfasst_get: level must be 0 or 1");
  }
  PFSH_CUDA(cudaMemcpyAsync(out, src, st * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return PFSH_OK;
}
