// Shared-memory Stockham FFT used by the longitude transforms.
//
// A transform of length N is a sequence of passes; the pass with radix R
// after sub-transform size Ns reads x[j + r N/R] (r < R), multiplies by the
// twiddles exp(-+2 pi i k r / (Ns R)), k = j mod Ns, does an R-point DFT in
// registers and writes y[(j/Ns) Ns R + k + q Ns] (q < R).  Radices 8 and 16
// are done in registers as 2x4 and 4x4 with their internal twiddles, so the
// common lengths take 3 or 4 passes (768 = 16*16*3).  For the grid sizes of
// the workloads the radix list is a template parameter, which turns all
// index arithmetic into constants; any other length (prime factors <= 61)
// takes the run-time path.  Shared-memory element e lives at e + e/16 so
// that the stride-R stores of the first passes do not serialise on banks.
#pragma once

#include "internal.cuh"

namespace pfsh {

struct FftArgs {
  int N, npass;
  int full;                // offset of the full-circle table exp(-2 pi i e/N), e < N
  int radix[kMaxPasses];
};

__device__ __forceinline__ int sidx(int e) { return e + (e >> 4); }
__host__ __device__ __forceinline__ int padded(int N) { return N + (N >> 4) + 1; }

template <typename C> __device__ __forceinline__ C twiddle(const C *tw, int e, bool inv) {
  C w = tw[e];
  if (inv) w.y = -w.y;
  return w;
}

template <typename C> __device__ __forceinline__ C rot_i(C a, bool inv) {
  // multiply by -i (forward) or +i (inverse)
  C r;
  if (inv) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

template <typename C> __device__ __forceinline__ void dft4(C &a0, C &a1, C &a2, C &a3, bool inv) {
  const C s02 = a0 + a2, d02 = a0 - a2, s13 = a1 + a3, d13 = a1 - a3;
  const C r = rot_i(d13, inv);          // -i (a1 - a3) forward
  a0 = s02 + s13;
  a2 = s02 - s13;
  a1 = d02 + r;
  a3 = d02 - r;
}

// exp(-2 pi i e / 16) for e = 0..15 (cos, -sin); conjugated for the inverse
__device__ __forceinline__ double c16(int e) {
  const double t[16] = {1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                        0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
                        -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173,
                        0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613};
  return t[e & 15];
}
__device__ __forceinline__ double s16(int e) { return c16(e + 12); }   // sin(2 pi e / 16)

template <typename C> __device__ __forceinline__ C w16(C a, int e, bool inv) {
  typedef decltype(a.x) R;
  const R c = (R)c16(e), s = inv ? (R)s16(e) : -(R)s16(e);
  C r;
  r.x = a.x * c - a.y * s;
  r.y = a.x * s + a.y * c;
  return r;
}

template <int R, typename C> __device__ __forceinline__ void butterfly(C *v, bool inv) {
  typedef decltype(v[0].x) Rt;
  if constexpr (R == 2) {
    const C a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  } else if constexpr (R == 3) {
    const Rt c = (Rt)-0.5;
    const Rt s = inv ? (Rt)0.86602540378443864676 : (Rt)-0.86602540378443864676;
    const C t = v[1] + v[2], u = v[1] - v[2];
    const C base = v[0] + c * t;
    C su;
    su.x = -s * u.y;
    su.y = s * u.x;
    v[0] = v[0] + t;
    v[1] = base + su;
    v[2] = base - su;
  } else if constexpr (R == 4) {
    dft4(v[0], v[1], v[2], v[3], inv);
  } else if constexpr (R == 5) {
    // X_q = sum_r v_r W5^{rq}; cos/sin of 2 pi/5 and 4 pi/5
    const Rt c1 = (Rt)0.30901699437494742410, c2 = (Rt)-0.80901699437494742410;
    const Rt s1 = inv ? (Rt)0.95105651629515357212 : (Rt)-0.95105651629515357212;
    const Rt s2 = inv ? (Rt)0.58778525229247312917 : (Rt)-0.58778525229247312917;
    const C a = v[1] + v[4], b = v[1] - v[4], c = v[2] + v[3], d = v[2] - v[3];
    const C t1 = v[0] + c1 * a + c2 * c, t2 = v[0] + c2 * a + c1 * c;
    C u1, u2;   // i (s1 b + s2 d), i (s2 b - s1 d)
    u1.x = -(s1 * b.y + s2 * d.y);
    u1.y = s1 * b.x + s2 * d.x;
    u2.x = -(s2 * b.y - s1 * d.y);
    u2.y = s2 * b.x - s1 * d.x;
    v[0] = v[0] + a + c;
    v[1] = t1 + u1;
    v[4] = t1 - u1;
    v[2] = t2 + u2;
    v[3] = t2 - u2;
  } else if constexpr (R == 8) {
    // n = q + 2r, k = s + 4t: U[q][s] = DFT4_r(v[q+2r])[s] W8^{qs}; X[s+4t] = DFT2_q
    C u0[4] = {v[0], v[2], v[4], v[6]}, u1[4] = {v[1], v[3], v[5], v[7]};
    dft4(u0[0], u0[1], u0[2], u0[3], inv);
    dft4(u1[0], u1[1], u1[2], u1[3], inv);
#pragma unroll
    for (int s = 1; s < 4; ++s) u1[s] = w16(u1[s], 2 * s, inv);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      v[s] = u0[s] + u1[s];
      v[s + 4] = u0[s] - u1[s];
    }
  } else if constexpr (R == 16) {
    // n = q + 4r, k = s + 4t: U[q][s] = DFT4_r(v[q+4r])[s] W16^{qs}; X[s+4t] = DFT4_q
    C u[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      u[q][0] = v[q];
      u[q][1] = v[q + 4];
      u[q][2] = v[q + 8];
      u[q][3] = v[q + 12];
      dft4(u[q][0], u[q][1], u[q][2], u[q][3], inv);
#pragma unroll
      for (int s = 1; s < 4; ++s)
        if (q) u[q][s] = w16(u[q][s], q * s, inv);
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      C a0 = u[0][s], a1 = u[1][s], a2 = u[2][s], a3 = u[3][s];
      dft4(a0, a1, a2, a3, inv);
      v[s] = a0;
      v[s + 4] = a1;
      v[s + 8] = a2;
      v[s + 12] = a3;
    }
  }
}

// The five products of the grid stage at one point (packed north/south rows).
template <typename C, typename Rl>
__device__ __forceinline__ void grid_products(const C &eta, const C &php, const C &U, const C &V, Rl inv, Rl h,
                                              C (&o)[5]) {
  const Rl Ui = U.x * inv, Us = U.y * inv, Vi = V.x * inv, Vs = V.y * inv;
  o[0] = mk<C>(eta.x * Ui, eta.y * Us);
  o[1] = mk<C>(eta.x * Vi, eta.y * Vs);
  o[2] = mk<C>(php.x * Ui, php.y * Us);
  o[3] = mk<C>(php.x * Vi, php.y * Vs);
  o[4] = mk<C>((U.x * U.x + V.x * V.x) * h, (U.y * U.y + V.y * V.y) * h);
}

// Twiddles are stored per pass: the pass with radix R after sub-transform
// size Ns owns R*Ns entries, entry r*Ns + k = exp(-2 pi i k r / (Ns R)), so
// the lanes of a warp (consecutive k) read consecutive entries.

// one compile-time pass over nfft transforms (padded stride between transforms)
template <int R, int Ns, int N, int OFF, typename C>
__device__ __forceinline__ void pass_ct(const C *__restrict__ x, C *__restrict__ y, int nfft,
                                        const C *__restrict__ tw, bool inv) {
  constexpr int NR = N / R;
  const int NP = padded(N);
  const int total = nfft * NR;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int fi = t / NR, j = t - fi * NR;
    const int k = j % Ns, idx = (j / Ns) * (Ns * R) + k;
    const C *xs = x + fi * NP;
    C *ys = y + fi * NP;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      C a = xs[sidx(j + r * NR)];
      if (Ns > 1 && r > 0) a = cmul(a, twiddle(tw, OFF + r * Ns + k, inv));
      v[r] = a;
    }
    butterfly<R>(v, inv);
#pragma unroll
    for (int q = 0; q < R; ++q) ys[sidx(idx + q * Ns)] = v[q];
  }
  __syncthreads();
}

// The first pass of an inverse grid-stage transform whose entries e with
// T < e < N - T are zero: they are neither stored nor read.
template <int R, int N, typename C>
__device__ __forceinline__ void pass_first_pruned(const C *__restrict__ x, C *__restrict__ y, int nfft, int T) {
  constexpr int NR = N / R;
  const int NP = padded(N);
  const int total = nfft * NR;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int fi = t / NR, j = t - fi * NR;
    const C *xs = x + fi * NP;
    C *ys = y + fi * NP;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = j + r * NR;
      v[r] = (e <= T || e >= N - T) ? xs[sidx(e)] : mk<C>(0.0, 0.0);
    }
    butterfly<R>(v, true);
#pragma unroll
    for (int q = 0; q < R; ++q) ys[sidx(j * R + q)] = v[q];
  }
  __syncthreads();
}

// The last pass of the 4 inverse grid-stage transforms (eta, Phi', U, V)
// fused with the grid products: one thread takes the same butterfly of all
// four rows (one twiddle load for the four), forms the five products at its
// R output points and stores them as the 5 rows y of the forward transform.
template <int R, int Ns, int N, int OFF, typename C, typename Rl>
__device__ __forceinline__ void pass_last_products(const C *__restrict__ x, C *__restrict__ y,
                                                   const C *__restrict__ tw, Rl inv, Rl h) {
  constexpr int NR = N / R;
  const int NP = padded(N);
  for (int j = threadIdx.x; j < NR; j += blockDim.x) {
    const int k = j % Ns, idx = (j / Ns) * (Ns * R) + k;
    C w[R];
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = Ns > 1 ? twiddle(tw, OFF + r * Ns + k, true) : mk<C>(1.0, 0.0);
    C v[4][R];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C a = x[f * NP + sidx(j + r * NR)];
        if (Ns > 1 && r > 0) a = cmul(a, w[r]);
        v[f][r] = a;
      }
      butterfly<R>(v[f], true);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      C pr[5];
      grid_products<C, Rl>(v[0][q], v[1][q], v[2][q], v[3][q], inv, h, pr);
#pragma unroll
      for (int p = 0; p < 5; ++p) y[p * NP + sidx(idx + q * Ns)] = pr[p];
    }
  }
  __syncthreads();
}

// inverse transforms of the 4 grid-stage rows with the products fused into
// the last pass (returns the buffer holding the 5 product rows)
template <int N, int Ns, int OFF, int... Rs> struct PassListF;
template <int N, int Ns, int OFF, int R> struct PassListF<N, Ns, OFF, R> {
  template <typename C, typename Rl>
  static __device__ __forceinline__ C *run(C *a, C *b, int, const C *tw, Rl inv, Rl h) {
    pass_last_products<R, Ns, N, OFF>(a, b, tw, inv, h);
    return b;
  }
};
template <int N, int Ns, int OFF, int R, int R2, int... Rs> struct PassListF<N, Ns, OFF, R, R2, Rs...> {
  template <typename C, typename Rl>
  static __device__ __forceinline__ C *run(C *a, C *b, int T, const C *tw, Rl inv, Rl h) {
    if constexpr (Ns == 1)
      pass_first_pruned<R, N>(a, b, 4, T);
    else
      pass_ct<R, Ns, N, OFF>(a, b, 4, tw, true);
    return PassListF<N, Ns * R, OFF + R * Ns, R2, Rs...>::run(b, a, T, tw, inv, h);
  }
};

template <int N, int Ns, int OFF, int... Rs> struct PassList;
template <int N, int Ns, int OFF> struct PassList<N, Ns, OFF> {
  template <typename C> static __device__ __forceinline__ C *run(C *a, C *, int, const C *, bool) { return a; }
};
template <int N, int Ns, int OFF, int R, int... Rs> struct PassList<N, Ns, OFF, R, Rs...> {
  template <typename C> static __device__ __forceinline__ C *run(C *a, C *b, int nfft, const C *tw, bool inv) {
    pass_ct<R, Ns, N, OFF>(a, b, nfft, tw, inv);
    return PassList<N, Ns * R, OFF + R * Ns, Rs...>::run(b, a, nfft, tw, inv);
  }
};

// the same pass list with the first pass pruned (inverse, Ns = 1: no twiddles)
template <int N, int R, int... Rs> struct PassListP {
  template <typename C> static __device__ __forceinline__ C *run(C *a, C *b, int nfft, int T, const C *tw) {
    pass_first_pruned<R, N>(a, b, nfft, T);
    return PassList<N, R, R, Rs...>::run(b, a, nfft, tw, true);
  }
};

template <int N_, int... Rs> struct ShapeCT {
  static constexpr bool kCT = true;
  static __host__ __device__ int n(const FftArgs &) { return N_; }
  template <typename C, typename Rl>
  static __device__ __forceinline__ C *inverse_products(C *a, C *b, int T, const C *tw, Rl inv, Rl h) {
    return PassListF<N_, 1, 0, Rs...>::run(a, b, T, tw, inv, h);
  }
  template <typename C>
  static __device__ __forceinline__ C *run(const FftArgs &, C *a, C *b, int nfft, const C *tw, bool inv) {
    return PassList<N_, 1, 0, Rs...>::run(a, b, nfft, tw, inv);
  }
  // inverse transforms whose entries T < e < N - T are zero (never read)
  template <typename C>
  static __device__ __forceinline__ C *inverse_pruned(C *a, C *b, int nfft, int T, const C *tw) {
    return PassListP<N_, Rs...>::run(a, b, nfft, T, tw);
  }
};

// run-time path: any length with prime factors <= 61
struct ShapeRT {
  static constexpr bool kCT = false;
  static __host__ __device__ int n(const FftArgs &f) { return f.N; }
  template <typename C>
  static __device__ C *run(const FftArgs &f, C *a, C *b, int nfft, const C *tw, bool inv) {
    const int N = f.N, NP = padded(N);
    int Ns = 1, off = 0;
    for (int p = 0; p < f.npass; ++p) {
      const int R = f.radix[p];
      const int NR = N / R;
      const int total = nfft * NR;
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int fi = t / NR, j = t - fi * NR;
        const C *x = a + fi * NP;
        C *y = b + fi * NP;
        const int k = j % Ns;
        const int idx = (j / Ns) * Ns * R + k;
        if (R == 4 || R == 2 || R == 3) {
          C v[4];
          for (int r = 0; r < R; ++r) {
            C w = x[sidx(j + r * NR)];
            if (r) w = cmul(w, twiddle(tw, off + r * Ns + k, inv));
            v[r] = w;
          }
          if (R == 4) butterfly<4>(v, inv);
          else if (R == 2) butterfly<2>(v, inv);
          else butterfly<3>(v, inv);
          for (int q = 0; q < R; ++q) y[sidx(idx + q * Ns)] = v[q];
        } else {
          for (int q = 0; q < R; ++q) {
            C acc = mk<C>(0.0, 0.0);
            for (int r = 0; r < R; ++r) {
              C v = x[sidx(j + r * NR)];
              if (r) v = cmul(v, twiddle(tw, off + r * Ns + k, inv));
              // W_R^{rq} = entry (r q mod R) * (N/R) of the last-pass layout:
              // use the full-circle table that follows the pass tables
              const int e = (r * q) % R;
              acc = acc + (e ? cmul(v, twiddle(tw, f.full + e * NR, inv)) : v);
            }
            y[sidx(idx + q * Ns)] = acc;
          }
        }
      }
      __syncthreads();
      C *tmp = a;
      a = b;
      b = tmp;
      off += R * Ns;
      Ns *= R;
    }
    return a;
  }
};

// lengths with a compile-time radix list
typedef ShapeCT<48, 16, 3> Shape48;
typedef ShapeCT<96, 16, 2, 3> Shape96;
typedef ShapeCT<192, 16, 4, 3> Shape192;
typedef ShapeCT<384, 16, 8, 3> Shape384;
typedef ShapeCT<768, 16, 16, 3> Shape768;
typedef ShapeCT<1536, 16, 16, 2, 3> Shape1536;
typedef ShapeCT<1920, 16, 8, 3, 5> Shape1920;
typedef ShapeCT<3840, 16, 16, 3, 5> Shape3840;

// Block-wide means of NF complex row sums (each thread passes its partial
// sums); `scratch` holds at least nwarps * NF elements and is free until the
// closing barrier.  Called by every thread of a block.
template <typename C, int NF>
__device__ __forceinline__ void block_means(decltype(C().x) (&sx)[NF], decltype(C().x) (&sy)[NF], int N,
                                            C *scratch, C (&mean)[NF]) {
  typedef decltype(C().x) R;
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      sx[f] += __shfl_xor_sync(0xffffffffu, sx[f], d);
      sy[f] += __shfl_xor_sync(0xffffffffu, sy[f], d);
    }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int f = 0; f < NF; ++f) scratch[warp * NF + f] = mk<C>(sx[f], sy[f]);
  __syncthreads();
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    R ax = (R)0, ay = (R)0;
    for (int w = 0; w < nw; ++w) {
      ax += scratch[w * NF + f].x;
      ay += scratch[w * NF + f].y;
    }
    mean[f] = mk<C>(ax / (R)N, ay / (R)N);
  }
  __syncthreads();
}

// Hemispheric sums and differences of the 5 forward-transformed product rows
// Z, weighted by w_j, into H[m][parity][j][b*5 + f] for m <= T (with the row
// mean restored at wavenumber 0 when `center`).  Called by every thread.
template <typename C, typename Rl>
__device__ __forceinline__ void grid_unpack(const C *Z, int N, int NP, int T, int j, int nlat, int colsH, int b,
                                            const Rl *__restrict__ rowf, C *__restrict__ H, bool center) {
  const Rl half = (Rl)0.5 / (Rl)N;
  const Rl wj = rowf[2 * j + 1];
  const int nh = nlat / 2;
  for (int t = threadIdx.x; t < 5 * (T + 1); t += blockDim.x) {
    const int m = t / 5, fld = t - 5 * m;   // consecutive threads: the 5 fields of one m
    const C *z = Z + fld * NP;
    C zm = z[sidx(m)];
    C zc = cconj(z[sidx(m == 0 ? 0 : N - m)]);
    if (center && m == 0) {                 // the row mean taken out before the transform
      const C dc = (Rl)N * z[NP - 1];
      zm = zm + dc;
      zc = zc + cconj(dc);
    }
    C gn = half * (zm + zc);
    C gs = half * times_i(zc - zm);
    C he = wj * (gn + gs), ho = wj * (gn - gs);
    H[(((size_t)m * 2 + 0) * nh + j) * colsH + b * 5 + fld] = he;
    H[(((size_t)m * 2 + 1) * nh + j) * colsH + b * 5 + fld] = ho;
  }
  __syncthreads();
}

// Row means are taken out of the products before the forward transform and
// put back at wavenumber 0 in the unpack (kept in the last slot, NP - 1, of
// each transform of both ping-pong buffers, which the passes never touch):
// the last Stockham pass of radix R mixes wavenumbers j + q N/R, and with
// R = 5 (nlon = 1920, 3840) the rounding of a large zonal mean would land
// inside the retained band, where the derivatives of the assembly amplify
// it.  The products are formed twice (sums, then centred values) rather
// than re-reading and rewriting the five product rows.  Only when the leak
// would land inside the band (nlon / last radix <= T: `center`); otherwise
// the products are formed once.

// RHS grid stage for one latitude pair (j, nlat-1-j) of state b: 4 spectra
// (eta, Phi', U, V) -> inverse FFTs -> products
//   A1 = eta U/(1-mu^2), B1 = eta V/(1-mu^2), A2 = Phi' U/(1-mu^2),
//   B2 = Phi' V/(1-mu^2), E = (U^2+V^2)/(2(1-mu^2))
// -> forward FFTs -> hemispheric sums/differences weighted by w_j.
// F columns b*4 + f, H columns b*5 + f; smem holds 10 padded transforms.
// Called by every thread of a block.
template <typename Rl, typename Shape>
__device__ __forceinline__ void grid_rhs_body(const FftArgs &f, int T, int nlat, int B, int j, int b,
                                              const typename cpx<Rl>::t *__restrict__ F, const Rl *__restrict__ rowf,
                                              const typename cpx<Rl>::t *__restrict__ tw,
                                              typename cpx<Rl>::t *__restrict__ H, typename cpx<Rl>::t *smem,
                                              bool center) {
  typedef typename cpx<Rl>::t C;
  const int N = Shape::n(f), NP = padded(N);
  C *A = smem;            // 5 padded transforms
  C *Bf = A + 5 * NP;     // 5 padded transforms
  const int js = nlat - 1 - j;
  const int colsF = 4 * B, colsH = 5 * B;
  // compile-time shapes without the row-mean removal: no zero fill (the first
  // inverse pass never reads the wavenumbers above T) and the products fused
  // into the last inverse pass
  const bool fused = Shape::kCT && !center;
  if (!fused) {
    for (int t = threadIdx.x; t < 4 * NP; t += blockDim.x) A[t] = mk<C>(0.0, 0.0);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < 4 * (T + 1); t += blockDim.x) {
    const int m = t >> 2, fld = t & 3;     // consecutive threads: the 4 fields of one m
    C fn = F[((size_t)m * nlat + j) * colsF + b * 4 + fld];
    C fs = F[((size_t)m * nlat + js) * colsF + b * 4 + fld];
    C *z = A + fld * NP;
    if (m == 0) {
      z[0] = mk<C>(fn.x, fs.x);
    } else {
      z[sidx(m)] = mk<C>(fn.x - fs.y, fn.y + fs.x);
      z[sidx(N - m)] = mk<C>(fn.x + fs.y, -fn.y + fs.x);
    }
  }
  __syncthreads();
  const Rl inv = rowf[2 * j];                // 1/(1 - mu_j^2)
  const Rl h = (Rl)0.5 * inv;
  if constexpr (Shape::kCT) {
    if (fused) {
      C *o = Shape::inverse_products(A, Bf, T, tw, inv, h);
      C *Z = Shape::run(f, o, (o == A) ? Bf : A, 5, tw, false);
      grid_unpack<C, Rl>(Z, N, NP, T, j, nlat, colsH, b, rowf, H, false);
      return;
    }
  }
  C *g = Shape::run(f, A, Bf, 4, tw, true);
  C *o = (g == A) ? Bf : A;
  C mean[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) mean[q] = mk<C>(0.0, 0.0);
  if (center) {
    Rl sx[5], sy[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) sx[q] = sy[q] = (Rl)0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      const int e = sidx(k);
      C pr[5];
      grid_products<C, Rl>(g[e], g[NP + e], g[2 * NP + e], g[3 * NP + e], inv, h, pr);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        sx[q] += pr[q].x;
        sy[q] += pr[q].y;
      }
    }
    block_means<C, 5>(sx, sy, N, o, mean);
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const int e = sidx(k);
    C pr[5];
    grid_products<C, Rl>(g[e], g[NP + e], g[2 * NP + e], g[3 * NP + e], inv, h, pr);
#pragma unroll
    for (int q = 0; q < 5; ++q) o[q * NP + e] = pr[q] - mean[q];
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      o[q * NP + NP - 1] = mean[q];
      g[q * NP + NP - 1] = mean[q];
    }
  __syncthreads();
  C *Z = Shape::run(f, o, g, 5, tw, false);
  grid_unpack<C, Rl>(Z, N, NP, T, j, nlat, colsH, b, rowf, H, center);
}

// Unpack of nf forward-transformed product rows Z (stride NP) holding fields
// f0 .. f0+nf-1: the same arithmetic per entry as grid_unpack, no barrier.
template <typename C, typename Rl>
__device__ __forceinline__ void grid_unpack_range(const C *Z, int f0, int nf, int N, int NP, int T, int j, int nlat,
                                                  int colsH, int b, const Rl *__restrict__ rowf,
                                                  C *__restrict__ H, bool center) {
  const Rl half = (Rl)0.5 / (Rl)N;
  const Rl wj = rowf[2 * j + 1];
  const int nh = nlat / 2;
  for (int t = threadIdx.x; t < nf * (T + 1); t += blockDim.x) {
    const int m = t / nf, q = t - nf * m;
    const C *z = Z + q * NP;
    C zm = z[sidx(m)];
    C zc = cconj(z[sidx(m == 0 ? 0 : N - m)]);
    if (center && m == 0) {
      const C dc = (Rl)N * z[NP - 1];
      zm = zm + dc;
      zc = zc + cconj(dc);
    }
    C gn = half * (zm + zc);
    C gs = half * times_i(zc - zm);
    C he = wj * (gn + gs), ho = wj * (gn - gs);
    H[(((size_t)m * 2 + 0) * nh + j) * colsH + b * 5 + f0 + q] = he;
    H[(((size_t)m * 2 + 1) * nh + j) * colsH + b * 5 + f0 + q] = ho;
  }
}

// The same grid stage for long rows, in shared memory for 6 instead of 10
// padded transforms (slots S0..S5):
//   1. the 4 spectra into S0..S3, inverse-transformed two at a time with
//      S4/S5 as the ping-pong pair (the first pass skips the zero band
//      T < e < N - T on compile-time shapes);
//   2. the 5 products formed once, in place, into S0..S4 (every thread reads
//      the 4 rows at the entries it writes), row means taken out when
//      `center`;
//   3. product 4 transformed with S5 as its work buffer and unpacked, then
//      products 0/1 and 2/3 in pairs with S4/S5 as the work pair.
// Same arithmetic per element as grid_rhs_body.
template <typename Rl, typename Shape>
__device__ __forceinline__ void grid_rhs_body_long(const FftArgs &f, int T, int nlat, int B, int j, int b,
                                                   const typename cpx<Rl>::t *__restrict__ F,
                                                   const Rl *__restrict__ rowf,
                                                   const typename cpx<Rl>::t *__restrict__ tw,
                                                   typename cpx<Rl>::t *__restrict__ H, typename cpx<Rl>::t *smem,
                                                   bool center) {
  typedef typename cpx<Rl>::t C;
  const int N = Shape::n(f), NP = padded(N);
  C *S = smem;
  C *W = S + 4 * NP;
  const int js = nlat - 1 - j;
  const int colsF = 4 * B, colsH = 5 * B;
  if constexpr (!Shape::kCT) {
    for (int t = threadIdx.x; t < 4 * NP; t += blockDim.x) S[t] = mk<C>(0.0, 0.0);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < 4 * (T + 1); t += blockDim.x) {
    const int m = t >> 2, fld = t & 3;     // consecutive threads: the 4 fields of one m
    C *z = S + fld * NP;
    C fn = F[((size_t)m * nlat + j) * colsF + b * 4 + fld];
    C fs = F[((size_t)m * nlat + js) * colsF + b * 4 + fld];
    if (m == 0) {
      z[0] = mk<C>(fn.x, fs.x);
    } else {
      z[sidx(m)] = mk<C>(fn.x - fs.y, fn.y + fs.x);
      z[sidx(N - m)] = mk<C>(fn.x + fs.y, -fn.y + fs.x);
    }
  }
  __syncthreads();
#pragma unroll
  for (int pr = 0; pr < 4; pr += 2) {
    C *a = S + pr * NP;
    C *r;
    if constexpr (Shape::kCT)
      r = Shape::inverse_pruned(a, W, 2, T, tw);
    else
      r = Shape::run(f, a, W, 2, tw, true);
    if (r != a) {
      for (int t = threadIdx.x; t < 2 * NP; t += blockDim.x) a[t] = r[t];
      __syncthreads();
    }
  }
  const Rl inv = rowf[2 * j];                // 1/(1 - mu_j^2)
  const Rl h = (Rl)0.5 * inv;
  Rl sx[5], sy[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) sx[q] = sy[q] = (Rl)0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const int e = sidx(k);
    C pr[5];
    grid_products<C, Rl>(S[e], S[NP + e], S[2 * NP + e], S[3 * NP + e], inv, h, pr);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      S[q * NP + e] = pr[q];
      sx[q] += pr[q].x;
      sy[q] += pr[q].y;
    }
  }
  C mean[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) mean[q] = mk<C>(0.0, 0.0);
  if (center) {
    block_means<C, 5>(sx, sy, N, W + NP, mean);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      const int e = sidx(k);
#pragma unroll
      for (int q = 0; q < 5; ++q) S[q * NP + e] = S[q * NP + e] - mean[q];
    }
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) S[q * NP + NP - 1] = mean[q];
    W[2 * NP - 1] = mean[4];
  }
  __syncthreads();
  const C *Z = Shape::run(f, W, W + NP, 1, tw, false);
  grid_unpack_range<C, Rl>(Z, 4, 1, N, NP, T, j, nlat, colsH, b, rowf, H, center);
  __syncthreads();
#pragma unroll
  for (int pr = 0; pr < 4; pr += 2) {
    if (threadIdx.x == 0) {
      W[NP - 1] = mean[pr];
      W[2 * NP - 1] = mean[pr + 1];
    }
    __syncthreads();
    Z = Shape::run(f, S + pr * NP, W, 2, tw, false);
    grid_unpack_range<C, Rl>(Z, pr, 2, N, NP, T, j, nlat, colsH, b, rowf, H, center);
    __syncthreads();
  }
}

// Radix list of the compile-time shape serving N (must match the typedefs
// above); false for lengths that take the run-time path.
inline bool ct_radix_list(int N, int *r, int *np) {
  static const int lists[][6] = {{48, 16, 3}, {96, 16, 2, 3}, {192, 16, 4, 3}, {384, 16, 8, 3}, {768, 16, 16, 3},
                                 {1536, 16, 16, 2, 3}, {1920, 16, 8, 3, 5}, {3840, 16, 16, 3, 5}};
  for (const auto &l : lists)
    if (l[0] == N) {
      int k = 0;
      for (int i = 1; i < 6 && l[i]; ++i) r[k++] = l[i];
      *np = k;
      return true;
    }
  return false;
}

// Calls f.template operator()<Shape>() with the shape serving length N.
template <typename Fn> int with_shape(int N, Fn &&fn) {
  switch (N) {
    case 48: return fn.template operator()<Shape48>();
    case 96: return fn.template operator()<Shape96>();
    case 192: return fn.template operator()<Shape192>();
    case 384: return fn.template operator()<Shape384>();
    case 768: return fn.template operator()<Shape768>();
    case 1536: return fn.template operator()<Shape1536>();
    case 1920: return fn.template operator()<Shape1920>();
    case 3840: return fn.template operator()<Shape3840>();
    default: return fn.template operator()<ShapeRT>();
  }
}

}  // namespace pfsh
