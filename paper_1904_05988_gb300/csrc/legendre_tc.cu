// Legendre contractions per order m on tcgen05 tensor cores (the discrete
// Legendre transform of Section 3) with bf16 operands and fp32 accumulation,
// optionally on split operands: two parts, hi*hi + hi*lo + lo*hi ("3xBF16",
// about 16 bits of each operand), or three, x = hi + mid + lo with the six
// products of the parts whose exponents sum above 2^-24 ("6xBF16", about 24
// bits: fp32 accuracy on tensor cores).
//
// Both directions are GEMMs with the 128 real columns of a CTA (re/im of the
// fields of a batch) as the MMA M dimension, so every accumulator row is one
// column and the epilogue writes consecutive columns from consecutive lanes:
//   synthesis  D_p[c][j] = sum_k X[m, n=m+2k+p][c] P_n^m(mu_j)   (K = degree)
//   analysis   D_p[c][i] = sum_j H_p[m][j][c] P_{n=m+2i+p}^m(mu_j) (K = latitude)
// with p the parity of n-m.  Synthesis combines F(+mu) = D_0 + D_1 and
// F(-mu) = D_0 - D_1; the weights w_j are already inside H.
//
// Operands live in shared memory in the canonical K-major no-swizzle layout
// (see tc.cuh).  The Legendre table side (B operand) is stored in global
// memory as ready-made shared-memory images, one per (m, row tile, parity,
// K chunk of <= 64), bf16 hi followed by bf16 lo, and is fetched with one
// bulk TMA copy per chunk; the activation side (A operand) is read as fp32
// (column pairs, float2) by the eight warps of the CTA, split into bf16
// hi/lo and stored to shared memory.  Two stages overlap the conversion of
// chunk q+1 with the MMAs of chunk q.  One thread issues the MMAs;
// accumulators for both parities live in TMEM (2 x N <= 512 columns) and are
// drained by both warpgroups (a warp reads the 32 TMEM lanes of its quadrant,
// the two warpgroups take alternate 16-column groups).  Every wait is
// bounded; on a timeout the status word records ST_TIMEOUT and the CTA winds
// down.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.cuh"
#include "tc.cuh"

namespace pfsh {

namespace {

constexpr int MROWS = 128;  // MMA M: real columns per CTA
// max K extent of one chunk for NS split parts (three-part images are halved
// in K so that two stages of both operands fit in shared memory)
__host__ __device__ constexpr int kc_of(int ns) { return ns == 3 ? 32 : 64; }

// the bf16/fp16 part products summed per K step for NS parts (a part, b part),
// largest first
__host__ __device__ constexpr int n_products(int ns) { return ns == 1 ? 1 : ns == 2 ? 3 : 6; }
__device__ constexpr int kProdA[6] = {0, 0, 1, 0, 2, 1};
__device__ constexpr int kProdB[6] = {0, 1, 0, 2, 0, 1};

// x split into NS 16-bit parts, part k = round(x - parts 0..k-1)
template <int NS, bool FP16>
__device__ __forceinline__ void split_parts(float x, uint16_t (&out)[NS]) {
  float r = x;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (FP16) {
      const __half h = __float2half_rn(r);
      out[k] = __half_as_ushort(h);
      r -= __half2float(h);
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(r);
      out[k] = __bfloat16_as_ushort(h);
      r -= __bfloat162float(h);
    }
  }
}

constexpr int NTHREADS = 256;

// At most 128 registers per thread (the analysis needs 147 unbounded, with no
// spill at 128): a CTA then leaves room in the register file for a coarse-
// chain block on the same SM, so the Step B transforms overlap the chain
// better (measured: 197 -> 202 iterations/s, 3xBF16, T255/T127, 32 slices).
template <int NS, bool FP16, bool ANALYSIS>
__global__ void __launch_bounds__(NTHREADS, 2)
    k_legendre_tc(int T, int nlat, int cols_real, int ntiles, const float *__restrict__ act,
                  const uint8_t *__restrict__ img, const TcChunk *__restrict__ chunks,
                  const TcWork *__restrict__ work, int Nmax, float *__restrict__ out, int *status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int nh = nlat / 2;
  const int cb = blockIdx.x, tile = blockIdx.y, m = blockIdx.z;
  const TcWork wk = work[m * ntiles + tile];
  if (wk.nchunks == 0) return;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = wk.N;
  constexpr int KC = kc_of(NS);
  const uint32_t a_half = MROWS * KC * 2;            // bytes of one A image part
  const uint32_t a_bytes = a_half * NS;
  const uint32_t b_half_max = (uint32_t)Nmax * KC * 2;
  const uint32_t b_bytes = b_half_max * NS;
  uint8_t *stA[2] = {smem, smem + a_bytes + b_bytes};
  uint8_t *stB[2] = {smem + a_bytes, smem + 2 * a_bytes + b_bytes};
  uint64_t *bars = (uint64_t *)(smem + 2 * (a_bytes + b_bytes));
  uint64_t *full = bars, *done = bars + 2, *fin = bars + 4;
  uint32_t *tmem_slot = (uint32_t *)(bars + 5);

  uint32_t ncols = 32;
  while (ncols < (uint32_t)(2 * N)) ncols <<= 1;
  if (tid == 0) {
    tc::mbar_init(&full[0], 1);
    tc::mbar_init(&full[1], 1);
    tc::mbar_init(&done[0], 1);
    tc::mbar_init(&done[1], 1);
    tc::mbar_init(fin, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, ncols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  const int m_len = T + 2 - m;          // degrees n = m .. T+1
  const size_t eo = (size_t)eoff(T, m);

  // split one item (columns r, r+1 x 8 consecutive K from k0) into NS parts
  // and store them in the parts of the A image A (tile K extent KL)
  auto store_item = [&](uint8_t *A, int r, int k0, int KL, const float2 (&v)[8]) {
    uint16_t p0[8][NS], p1[8][NS];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      split_parts<NS, FP16>(v[i].x, p0[i]);
      split_parts<NS, FP16>(v[i].y, p1[i]);
    }
    const uint32_t off0 = tc::tile_offset(r, k0, KL), off1 = tc::tile_offset(r + 1, k0, KL);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      uint8_t *Ak = A + (size_t)k * a_half;
      *(uint4 *)(Ak + off0) = make_uint4(p0[0][k] | (uint32_t)p0[1][k] << 16, p0[2][k] | (uint32_t)p0[3][k] << 16,
                                         p0[4][k] | (uint32_t)p0[5][k] << 16, p0[6][k] | (uint32_t)p0[7][k] << 16);
      *(uint4 *)(Ak + off1) = make_uint4(p1[0][k] | (uint32_t)p1[1][k] << 16, p1[2][k] | (uint32_t)p1[3][k] << 16,
                                         p1[4][k] | (uint32_t)p1[5][k] << 16, p1[6][k] | (uint32_t)p1[7][k] << 16);
    }
  };
  // MMAs of one chunk (stage A, stage B, K extent KL, parity p) into TMEM
  auto issue_mmas = [&](const uint8_t *A, const uint8_t *Bimg, const TcChunk &ch) {
    const int KL = ch.klen;
    const uint32_t idesc = tc::make_idesc(MROWS, N, FP16);
    const uint32_t sbo = 16u * KL;
    const uint32_t b_half = (uint32_t)N * KL * 2;
    const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(Bimg);
    const uint32_t d = tmem + (uint32_t)(ch.p * N);
    for (int ks = 0; ks < KL / 16; ++ks) {
#pragma unroll
      for (int q = 0; q < n_products(NS); ++q) {
        const uint32_t acc = (ch.kstart == 0 && ks == 0 && q == 0) ? 0u : 1u;
        const uint64_t ad = tc::make_desc(a0 + kProdA[q] * a_half + ks * 256, 128, sbo);
        const uint64_t bd = tc::make_desc(b0 + kProdB[q] * b_half + ks * 256, 128, sbo);
        tc::mma_f16(d, ad, bd, idesc, acc);
      }
    }
  };
  // activation items of one chunk (two adjacent columns x 8 consecutive K,
  // loaded as float2) into registers; zeros outside the tile
  constexpr int MAXIT = (MROWS / 2) * (KC / 8) / NTHREADS;
  auto load_chunk = [&](int q, float2 (&v)[MAXIT][8]) {
    const TcChunk ch = chunks[wk.first + q];
    const int nit = (MROWS / 2) * (ch.klen >> 3);
#pragma unroll
    for (int u = 0; u < MAXIT; ++u) {
      const int it = tid + u * NTHREADS;
      const int rp = it & (MROWS / 2 - 1), g = it >> 6;
      const int c = cb * MROWS + 2 * rp;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = ch.kstart + g * 8 + i;
        v[u][i] = make_float2(0.f, 0.f);
        if (it < nit && c < cols_real) {
          if (!ANALYSIS) {
            const int noff = 2 * k + ch.p;      // n - m
            if (noff < m_len) v[u][i] = *(const float2 *)(act + (eo + noff) * cols_real + c);
          } else {
            if (k < nh) v[u][i] = *(const float2 *)(act + (((size_t)m * 2 + ch.p) * nh + k) * cols_real + c);
          }
        }
      }
    }
  };
  // stage chunk q (registers v) into shared memory and issue its MMAs
  auto produce = [&](int q, float2 (&v)[MAXIT][8]) {
    const TcChunk ch = chunks[wk.first + q];
    const int s = q & 1, u2 = q >> 1;
    if (q >= 2) ok &= tc::mbar_wait(&done[s], (u2 - 1) & 1);
    const int KL = ch.klen;
    const uint32_t b_half = (uint32_t)N * KL * 2;
    if (tid == 0) {
      const uint32_t bytes = b_half * NS;
      tc::mbar_arrive_expect_tx(&full[s], bytes);
      tc::bulk_g2s(stB[s], img + ch.off, bytes, &full[s]);
    }
    const int nit = (MROWS / 2) * (KL >> 3);
#pragma unroll
    for (int uu = 0; uu < MAXIT; ++uu) {
      const int it = tid + uu * NTHREADS;
      if (it >= nit) continue;
      const int rp = it & (MROWS / 2 - 1), g = it >> 6;
      store_item(stA[s], 2 * rp, g * 8, KL, v[uu]);
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      ok &= tc::mbar_wait(&full[s], u2 & 1);
      tc::fence_after_sync();
      issue_mmas(stA[s], stB[s], ch);
      tc::mma_commit(&done[s]);
    }
  };
  if constexpr (ANALYSIS) {
    // analysis (K = latitudes, six chunks per CTA at T255): two register
    // sets, the loads of chunk q+1 in flight while chunk q is converted and
    // multiplied (unrolled by two so that both sets stay in registers)
    float2 va[MAXIT][8], vb[MAXIT][8];
    if (wk.nchunks > 0) load_chunk(0, va);
    for (int q = 0; q < wk.nchunks; q += 2) {
      if (q + 1 < wk.nchunks) load_chunk(q + 1, vb);
      produce(q, va);
      if (q + 1 < wk.nchunks) {
        if (q + 2 < wk.nchunks) load_chunk(q + 2, va);
        produce(q + 1, vb);
      }
    }
  } else {
    // synthesis (K = degrees of one parity, few chunks): each thread loads,
    // splits and stores its items of chunk q in turn (measured faster than
    // the two-set prefetch here: 31 vs 48 us at T255 with 16 states)
    for (int q = 0; q < wk.nchunks; ++q) {
      const TcChunk ch = chunks[wk.first + q];
      const int s = q & 1, u = q >> 1;
      if (q >= 2) ok &= tc::mbar_wait(&done[s], (u - 1) & 1);
      const int KL = ch.klen;
      const uint32_t b_half = (uint32_t)N * KL * 2;
      if (tid == 0) {
        const uint32_t bytes = b_half * NS;
        tc::mbar_arrive_expect_tx(&full[s], bytes);
        tc::bulk_g2s(stB[s], img + ch.off, bytes, &full[s]);
      }
      // produce the activation chunk: rows = 128 real columns, K = KL; one
      // item = two adjacent columns x 8 consecutive K, loaded as float2
      const int groups = KL >> 3;
      for (int it = tid; it < (MROWS / 2) * groups; it += NTHREADS) {
        const int rp = it & (MROWS / 2 - 1), g = it >> 6;
        const int r = 2 * rp, c = cb * MROWS + r;
        float2 v[8];
  #pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = ch.kstart + g * 8 + i;
          v[i] = make_float2(0.f, 0.f);
          if (c < cols_real) {
            if (!ANALYSIS) {
              const int noff = 2 * k + ch.p;      // n - m
              if (noff < m_len) v[i] = *(const float2 *)(act + (eo + noff) * cols_real + c);
            } else {
              if (k < nh) v[i] = *(const float2 *)(act + (((size_t)m * 2 + ch.p) * nh + k) * cols_real + c);
            }
          }
        }
        store_item(stA[s], r, g * 8, KL, v);
      }
      tc::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        ok &= tc::mbar_wait(&full[s], u & 1);
        tc::fence_after_sync();
        issue_mmas(stA[s], stB[s], ch);
        tc::mma_commit(&done[s]);
      }
    }
  }
  if (tid == 0) tc::mma_commit(fin);
  ok &= tc::mbar_wait(fin, 0);
  tc::fence_after_sync();

  // epilogue: lane = real column, TMEM column = row of the tile; warp w reads
  // the lanes of quadrant w % 4, warpgroup w / 4 takes every other 16 columns
  const int quad = warp & 3, wg = warp >> 2;
  const int c = cb * MROWS + quad * 32 + (tid & 31);
  const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
  for (int c0 = wg * 16; c0 < N; c0 += 32) {
    float v0[16], v1[16];
    tc::tmem_ld16(tl + c0, v0);
    tc::tmem_ld16(tl + N + c0, v1);
    if (c >= cols_real) continue;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int row = wk.row0 + c0 + i;
      if (c0 + i >= wk.nrows) break;
      if (!ANALYSIS) {
        out[((size_t)m * nlat + row) * cols_real + c] = v0[i] + v1[i];
        out[((size_t)m * nlat + (nlat - 1 - row)) * cols_real + c] = v0[i] - v1[i];
      } else {
        const int n0 = 2 * row;               // n - m of parity 0
        if (n0 < m_len) out[(eo + n0) * cols_real + c] = v0[i];
        if (n0 + 1 < m_len) out[(eo + n0 + 1) * cols_real + c] = v1[i];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
  if (!ok && tid == 0 && status) atomicExch(status, ST_TIMEOUT);
}

// Build the table images from the FP64 table: one block per chunk; NS parts,
// part k = round(P - parts 0..k-1) (the remainder carried in FP64).
template <int NS, bool FP16, bool ANALYSIS>
__global__ void k_build_images(int T, int nh, const double *__restrict__ P, const TcChunk *__restrict__ chunks,
                               uint8_t *__restrict__ img) {
  const TcChunk ch = chunks[blockIdx.x];
  const int N = ch.N, KL = ch.klen;
  const int m_len = T + 2 - ch.m;
  const size_t eo = (size_t)eoff(T, ch.m);
  uint8_t *base = img + ch.off;
  for (int e = threadIdx.x; e < N * KL; e += blockDim.x) {
    const int r = e / KL, k = e - r * KL;
    double v = 0.0;
    if (r < ch.nrows) {
      if (!ANALYSIS) {
        const int j = ch.row0 + r, noff = 2 * (ch.kstart + k) + ch.p;
        if (j < nh && noff < m_len) v = P[(eo + noff) * nh + j];
      } else {
        const int noff = 2 * (ch.row0 + r) + ch.p, j = ch.kstart + k;
        if (j < nh && noff < m_len) v = P[(eo + noff) * nh + j];
      }
    }
    const uint32_t off = tc::tile_offset(r, k, KL);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      uint16_t h;
      if (FP16) {
        const __half hh = __double2half(v);
        h = __half_as_ushort(hh);
        v -= (double)__half2float(hh);
      } else {
        const __nv_bfloat16 hh = __double2bfloat16(v);
        h = __bfloat16_as_ushort(hh);
        v -= (double)__bfloat162float(hh);
      }
      *(uint16_t *)(base + (size_t)q * N * KL * 2 + off) = h;
    }
  }
}

int round16(int x) { return (x + 15) & ~15; }

// host-side chunk lists for one direction
void plan_chunks(int T, int nh, bool analysis, int tile_mult, int ns, std::vector<TcChunk> &chunks,
                 std::vector<TcWork> &work, int &ntiles, int &Nmax, size_t &bytes) {
  const int KC = kc_of(ns);
  chunks.clear();
  work.clear();
  Nmax = 16;
  bytes = 0;
  int rows_total, tiles;
  if (!analysis) {
    rows_total = nh;                         // tiles over latitudes
  } else {
    rows_total = (T + 3) / 2;                // degree positions of parity 0 at m = 0
  }
  tiles = (rows_total + 255) / 256 * tile_mult;
  tiles = std::max(1, std::min(tiles, rows_total / 16));   // at least 16 rows per tile
  const int tsz = (rows_total + tiles - 1) / tiles;
  ntiles = tiles;
  for (int m = 0; m <= T; ++m) {
    const int Km = T + 2 - m;
    const int K0 = (Km + 1) / 2;
    for (int t = 0; t < tiles; ++t) {
      TcWork w{};
      w.first = (int)chunks.size();
      w.row0 = t * tsz;
      const int lim = analysis ? K0 : nh;
      w.nrows = std::max(0, std::min(tsz, lim - w.row0));
      w.N = round16(std::max(w.nrows, 1));
      if (w.nrows == 0) {
        w.nchunks = 0;
        work.push_back(w);
        continue;
      }
      Nmax = std::max(Nmax, w.N);
      for (int p = 0; p < 2; ++p) {
        const int Kext = analysis ? round16(nh) : (Km + 1 - p) / 2;
        if (Kext <= 0) continue;
        for (int k0 = 0; k0 < Kext; k0 += KC) {
          TcChunk c{};
          c.off = (long long)bytes;
          c.m = m;
          c.p = p;
          c.kstart = k0;
          c.klen = round16(std::min(KC, Kext - k0));
          c.N = w.N;
          c.row0 = w.row0;
          c.nrows = w.nrows;
          bytes += (size_t)c.N * c.klen * 2 * std::max(ns, 2);   // the parts (at least hi + lo)
          chunks.push_back(c);
        }
      }
      w.nchunks = (int)chunks.size() - w.first;
      work.push_back(w);
    }
  }
}

template <typename K>
int set_smem_attr(K kernel, size_t bytes) {
  return ensure_smem((const void *)kernel, bytes);
}

size_t tc_smem_bytes(int Nmax, int ns) {
  const size_t a = (size_t)MROWS * kc_of(ns) * 2 * ns;
  const size_t b = (size_t)Nmax * kc_of(ns) * 2 * ns;
  return 2 * (a + b) + 64 + 1024;
}

}  // namespace

// images, chunk and work lists of one direction and row tiling
// 16-bit operand parts of a tensor-core precision
static int ns_of(int prec) { return prec == PFSH_BF16X6 ? 3 : prec == PFSH_BF16X3 ? 2 : 1; }

static int tc_build_dir(sht_plan *p, int dir, int tile_mult, TcDir &d) {
  const bool fp16 = p->prec == PFSH_FP16;
  const int ns = ns_of(p->prec);
  std::vector<TcChunk> ch;
  std::vector<TcWork> wk;
  plan_chunks(p->T, p->nh, dir == 1, tile_mult, ns, ch, wk, d.ntiles, d.Nmax, d.img_bytes);
  d.nchunks = (int)ch.size();
  if (cudaMalloc(&d.img, d.img_bytes) != cudaSuccess || cudaMalloc(&d.chunks, ch.size() * sizeof(TcChunk)) ||
      cudaMalloc(&d.work, wk.size() * sizeof(TcWork))) {
    cudaGetLastError();
    return fail(PFSH_ENOMEM, "tensor-core table images");
  }
  p->device_bytes += d.img_bytes + ch.size() * sizeof(TcChunk) + wk.size() * sizeof(TcWork);
  PFSH_CUDA(cudaMemcpy(d.chunks, ch.data(), ch.size() * sizeof(TcChunk), cudaMemcpyHostToDevice));
  PFSH_CUDA(cudaMemcpy(d.work, wk.data(), wk.size() * sizeof(TcWork), cudaMemcpyHostToDevice));
  PFSH_CUDA(cudaMemset(d.img, 0, d.img_bytes));
  {
    PFSH_LAUNCH("k_build_images", 0);
    auto launch = [&](auto kern) { kern<<<d.nchunks, 256>>>(p->T, p->nh, p->d_P, d.chunks, d.img); };
    if (dir == 0) {
      if (fp16) launch(k_build_images<1, true, false>);
      else if (ns == 1) launch(k_build_images<1, false, false>);
      else if (ns == 2) launch(k_build_images<2, false, false>);
      else launch(k_build_images<3, false, false>);
    } else {
      if (fp16) launch(k_build_images<1, true, true>);
      else if (ns == 1) launch(k_build_images<1, false, true>);
      else if (ns == 2) launch(k_build_images<2, false, true>);
      else launch(k_build_images<3, false, true>);
    }
  }
  PFSH_CHECK_LAUNCH("k_build_images");
  return PFSH_OK;
}

static void tc_free_dir(sht_plan *p, TcDir &d) {
  if (d.img) cudaFree(d.img);
  if (d.chunks) cudaFree(d.chunks);
  if (d.work) cudaFree(d.work);
  const size_t held = d.img_bytes + (size_t)d.nchunks * sizeof(TcChunk) + (size_t)(p->T + 1) * d.ntiles * sizeof(TcWork);
  p->device_bytes -= std::min(p->device_bytes, held);
  d = TcDir{};
}

// ---------------------------------------------------------------------------
// Autotuner.  For each direction and launch width nb (column blocks of 128
// real columns), the configurations built for the plan are timed on the
// plan's workspace (CUDA events, 2 warm-up + 5 timed launches each) and the
// fastest is kept.  Results are cached per (T, nlat, precision, direction,
// nb) for the process and, when PFSH_TUNE_CACHE names a file, in that file
// (one JSON object per line), so plans of the same shape reuse them.
// PFSH_TC_TILES = 1 or 2 pins the row-tile multiplier instead.
// ---------------------------------------------------------------------------
using TuneKey = std::tuple<int, int, int, int, int>;   // T, nlat, prec, dir, nb
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tune;   // -> row-tile multiplier
static bool g_tune_loaded = false;

static void tune_cache_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = getenv("PFSH_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof line, f)) {
    int T, nlat, prec, dir, nb, mult;
    if (sscanf(line, "{\"T\": %d, \"nlat\": %d, \"prec\": %d, \"dir\": %d, \"nb\": %d, \"tile_mult\": %d",
               &T, &nlat, &prec, &dir, &nb, &mult) == 6 && (mult == 1 || mult == 2))
      g_tune[TuneKey(T, nlat, prec, dir, nb)] = mult;
  }
  fclose(f);
}

static void tune_cache_store(const TuneKey &k, int mult, const float us[kTcConfigs]) {
  g_tune[k] = mult;
  const char *path = getenv("PFSH_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"T\": %d, \"nlat\": %d, \"prec\": %d, \"dir\": %d, \"nb\": %d, \"tile_mult\": %d, "
             "\"us\": [%.2f, %.2f]}\n",
          std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), mult, us[0], us[1]);
  fclose(f);
}

template <int NS, bool FP16, bool AN>
static int launch_tc(const sht_plan *p, const TcDir &d, int cols, const float *act, float *out, cudaStream_t s,
                     const char *name);
static int launch_dir(const sht_plan *p, int dir, const TcDir &d, int cols, cudaStream_t s);

static int tc_time(const sht_plan *p, int dir, const TcDir &d, int cols, float *us) {
  cudaEvent_t e0, e1;
  PFSH_CUDA(cudaEventCreate(&e0));
  PFSH_CUDA(cudaEventCreate(&e1));
  int rc = PFSH_OK;
  for (int it = 0; it < 2 && !rc; ++it) rc = launch_dir(p, dir, d, cols, 0);
  cudaEventRecord(e0, 0);
  for (int it = 0; it < 5 && !rc; ++it) rc = launch_dir(p, dir, d, cols, 0);
  cudaEventRecord(e1, 0);
  float ms = 0.0f;
  if (!rc && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
    *us = ms * 1000.0f / 5.0f;
  else if (!rc)
    rc = fail(PFSH_ECUDA, "autotuner timing");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int tc_tables_build(sht_plan *p) {
  const char *pin = getenv("PFSH_TC_TILES");
  const int forced = pin && (pin[0] == '1' || pin[0] == '2') && pin[1] == 0 ? pin[0] - '0' : 0;
  // launch widths of this plan: up to max_batch complex columns
  const int nb_max = std::min(kTcMaxNb, (2 * p->max_batch + MROWS - 1) / MROWS);
  int rc;
  for (int dir = 0; dir < 2; ++dir) {
    // widths at which the small-batch kernels run instead never reach these kernels
    auto small = [&](int cols) { return dir == 0 ? small_synth(cols) : small_analysis(cols); };
    for (int i = 0; i < kTcMaxNb; ++i) p->tc_pick[dir][i] = 0;
    if (forced) {
      p->tc_mult[dir][0] = forced;
      if ((rc = tc_build_dir(p, dir, forced, p->tc[dir][0]))) return rc;
      continue;
    }
    p->tc_mult[dir][0] = 1;
    if ((rc = tc_build_dir(p, dir, 1, p->tc[dir][0]))) return rc;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_load();
    // timed width of nb column blocks: nb x 64 complex columns, within the workspace
    auto width = [&](int nb) { return std::min(p->max_batch, nb * MROWS / 2); };
    int need = 0;   // launch widths without a cached choice
    for (int nb = 1; nb <= nb_max; ++nb)
      if (!small(width(nb)) && !g_tune.count(TuneKey(p->T, p->nlat, p->prec, dir, nb))) ++need;
    bool want2 = false;
    for (int nb = 1; nb <= nb_max; ++nb) {
      auto it = g_tune.find(TuneKey(p->T, p->nlat, p->prec, dir, nb));
      if (it != g_tune.end() && it->second == 2) want2 = true;
    }
    if (need > 0 || want2) {
      p->tc_mult[dir][1] = 2;
      if ((rc = tc_build_dir(p, dir, 2, p->tc[dir][1]))) return rc;
      if (p->tc[dir][1].ntiles == p->tc[dir][0].ntiles) {   // too few rows to split further
        tc_free_dir(p, p->tc[dir][1]);
        p->tc_mult[dir][1] = 0;
      }
    }
    if (need > 0 && p->tc_mult[dir][1]) {
      PFSH_CUDA(cudaMemset(p->ws, 0, p->ws_bytes));
      for (int nb = 1; nb <= nb_max; ++nb) {
        const TuneKey key(p->T, p->nlat, p->prec, dir, nb);
        const int cols = width(nb);
        if (small(cols) || g_tune.count(key)) continue;
        float us[kTcConfigs] = {0.0f, 0.0f};
        for (int c = 0; c < kTcConfigs; ++c)
          if ((rc = tc_time(p, dir, p->tc[dir][c], cols, &us[c]))) return rc;
        tune_cache_store(key, us[1] < us[0] ? 2 : 1, us);
      }
    }
    bool uses2 = false;
    for (int nb = 1; nb <= kTcMaxNb; ++nb) {
      auto it = g_tune.find(TuneKey(p->T, p->nlat, p->prec, dir, std::min(nb, nb_max)));
      const int c = (it != g_tune.end() && it->second == 2 && p->tc_mult[dir][1]) ? 1 : 0;
      p->tc_pick[dir][nb - 1] = (unsigned char)c;
      uses2 |= c == 1;
    }
    if (!uses2 && p->tc_mult[dir][1]) {
      tc_free_dir(p, p->tc[dir][1]);
      p->tc_mult[dir][1] = 0;
    }
  }
  PFSH_CUDA(cudaDeviceSynchronize());
  return PFSH_OK;
}

void tc_tables_free(sht_plan *p) {
  for (int dir = 0; dir < 2; ++dir)
    for (int c = 0; c < kTcConfigs; ++c) {
      TcDir &d = p->tc[dir][c];
      if (d.img) cudaFree(d.img);
      if (d.chunks) cudaFree(d.chunks);
      if (d.work) cudaFree(d.work);
      d = TcDir{};
    }
}

int tc_tiles_used(const sht_plan *p, int dir, int nb) {
  if (!uses_tensor_cores(p->prec) || nb < 1) return 0;
  return p->tc[dir][p->tc_pick[dir][std::min(nb, kTcMaxNb) - 1]].ntiles;
}

template <int NS, bool FP16, bool AN>
static int launch_tc(const sht_plan *p, const TcDir &d, int cols, const float *act, float *out, cudaStream_t s,
                     const char *name) {
  const int cols_real = 2 * cols;
  const size_t smem = tc_smem_bytes(d.Nmax, NS);
  auto kern = k_legendre_tc<NS, FP16, AN>;
  int rc = set_smem_attr(kern, smem);
  if (rc) return rc;
  dim3 g((cols_real + MROWS - 1) / MROWS, d.ntiles, p->T + 1);
  {
    PFSH_LAUNCH(name, s);
    kern<<<g, NTHREADS, smem, s>>>(p->T, p->nlat, cols_real, d.ntiles, act, d.img, d.chunks, d.work, d.Nmax, out,
                              device_status());
  }
  PFSH_CHECK_LAUNCH(name);
  return PFSH_OK;
}

// one launch of direction dir with the row tiling d
static int launch_dir(const sht_plan *p, int dir, const TcDir &d, int cols, cudaStream_t s) {
  if (dir == 0) {
    const float *X = (const float *)p->X;
    float *F = (float *)p->F;
    switch (p->prec) {
      case PFSH_BF16: return launch_tc<1, false, false>(p, d, cols, X, F, s, "k_synth_bf16");
      case PFSH_FP16: return launch_tc<1, true, false>(p, d, cols, X, F, s, "k_synth_fp16");
      case PFSH_BF16X3: return launch_tc<2, false, false>(p, d, cols, X, F, s, "k_synth_bf16x3");
      case PFSH_BF16X6: return launch_tc<3, false, false>(p, d, cols, X, F, s, "k_synth_bf16x6");
      default: return fail(PFSH_EUNSUPPORTED, "synth_tc: precision");
    }
  }
  const float *H = (const float *)p->H;
  float *Y = (float *)p->Y;
  switch (p->prec) {
    case PFSH_BF16: return launch_tc<1, false, true>(p, d, cols, H, Y, s, "k_anal_bf16");
    case PFSH_FP16: return launch_tc<1, true, true>(p, d, cols, H, Y, s, "k_anal_fp16");
    case PFSH_BF16X3: return launch_tc<2, false, true>(p, d, cols, H, Y, s, "k_anal_bf16x3");
    case PFSH_BF16X6: return launch_tc<3, false, true>(p, d, cols, H, Y, s, "k_anal_bf16x6");
    default: return fail(PFSH_EUNSUPPORTED, "analysis_tc: precision");
  }
}

// the tiling the autotuner picked for this launch width
static const TcDir &tc_for(const sht_plan *p, int dir, int cols) {
  const int nb = std::min(kTcMaxNb, std::max(1, (2 * cols + MROWS - 1) / MROWS));
  return p->tc[dir][p->tc_pick[dir][nb - 1]];
}

int synth_tc(const sht_plan *p, int cols, cudaStream_t s) { return launch_dir(p, 0, tc_for(p, 0, cols), cols, s); }

int analysis_tc(const sht_plan *p, int cols, cudaStream_t s) { return launch_dir(p, 1, tc_for(p, 1, cols), cols, s); }

}  // namespace pfsh
