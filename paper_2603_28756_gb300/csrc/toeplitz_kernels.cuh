// The per-iteration hot path: R*R y as a zero-padded 2N x 2N FFT convolution with the
// point-spread kernel (Sec. 2.1, Eq. 9), fused with -R*g (Eq. 11), the qGGMRF prior
// gradient over the 26-neighbourhood (Eq. 5, Sec. 2.4) and the fast-gradient update with
// restart (Sec. 2, Eq. 6).
//
// Three passes per iteration, each one launch over every slice of a group:
//   pass 1  rows:    y = x_k + beta (x_k - x_{k-1}); real FFT of length 2N of each row (the
//                    upper N entries are the zero padding), written column-major
//                    spec[v][r], v = 0..N (half spectrum), r = 0..N-1 (nonzero rows only).
//   pass 2  columns: per column v, FFT of length 2N of the N nonzero rows, multiply by the
//                    real kernel spectrum, inverse FFT, keep the first N rows (the crop).
//                    The length-2N transforms are split into their even and odd halves, two
//                    length-N transforms each, so the zero padding and the crop cost nothing.
//   pass 3  rows:    inverse real FFT of each row, keep the first N columns -> K (*) y; then
//                    per voxel G = K(*)y - R*g + lambda grad Phi(y), x_{k+1} = y - G/L, and the
//                    FP64 partial sums the optimiser needs.
// A finalize kernel (one block) reduces the partials in a fixed order and advances the
// device-resident momentum state, so a whole run needs no host round trip.
//
// The intermediate spectrum is stored as FP32 complex, or (BF = true) as BF16 pairs with all
// arithmetic still in FP32: the storage halves and every transform accumulates in FP32.
#pragma once
#include <cuda_bf16.h>

#include "block_fft.cuh"
#include "fft.cuh"
#include "internal.h"

namespace tmbir {

// ---------------------------------------------------------------- spectrum storage
template <bool BF>
struct SpecIO;
template <>
struct SpecIO<false> {
  using T = float2;
  __device__ __forceinline__ static float2 ld(const T* p, size_t i) { return p[i]; }
  __device__ __forceinline__ static void st(T* p, size_t i, float2 v) { p[i] = v; }
};
template <>
struct SpecIO<true> {
  using T = __nv_bfloat162;
  __device__ __forceinline__ static float2 ld(const T* p, size_t i) { return __bfloat1622float2(p[i]); }
  __device__ __forceinline__ static void st(T* p, size_t i, float2 v) { p[i] = __float22bfloat162_rn(v); }
};
// In Iterate mode every pass checks the run's current storage phase and leaves when it is
// not its own, so the BF16 and FP32 variants can be enqueued back to back.
template <bool BF>
__device__ __forceinline__ bool skip_iter(const IterState* st) {
  return st->done || (st->bf16 != 0) != BF;
}

// ---------------------------------------------------------------- launch geometry
template <int N>
struct Geo {
  using F = typename FFTShape<N>::type;
  static constexpr int T = F::T, P = F::P, G = 32 / T;
  static constexpr int W = 4;           // warps per block
  static constexpr int THREADS = 32 * W;
  static constexpr int RB = W * G;      // rows per block in passes 1 and 3
  static constexpr int NB = N / RB;     // row blocks per slice
  static constexpr int LD = N + 4;      // row stride (complex) of the row-major staging buffer
  static constexpr int UNITS = W * G;   // (column, half) units per block in pass 2
  static constexpr int CPB = UNITS / 2; // columns per block in pass 2
  static constexpr size_t SM_FFT = (size_t)W * G * F::SMEM * sizeof(float2);
  static constexpr size_t SM_TB = (size_t)RB * LD * sizeof(float2);
  static constexpr size_t SM_Y = (size_t)3 * (RB + 2) * N * sizeof(float);
  static constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
  static constexpr size_t SM1 = cmax(SM_FFT, SM_TB);
  static constexpr size_t SM2 = SM_FFT;
  static constexpr size_t SM3 = cmax(SM1, SM_Y);
};

// ---------------------------------------------------------------- special-function unit helpers
__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpa(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/x for x >= 1 on the FMA pipe: integer seed then three Newton steps r <- r (2 - x r).
// Seed: the bit pattern of 1/x is about (253 + c) 2^23 - bits(x); c = 0.9 balances the seed
// error to within 5.2 % over every binade, and three quadratic steps bring it below 1e-7.
__device__ __forceinline__ float rcp_newton(float x) {
  float r = __int_as_float(0x7EF33333 - __float_as_int(x));
#pragma unroll
  for (int it = 0; it < 3; ++it) r = fmaf(r, fmaf(-x, r, 1.0f), r);
  return r;
}

// Packed FP32 pairs: one instruction computes both lanes of a float2 (sm_100 and later).
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Constants of the qGGMRF potential in the form the packed neighbour term uses.
struct PriorK {
  float2 half_qp;  // (q - p) / 2
  float2 qp_l2;    // (q - p) log2(1 / (c sigma))
  float2 p, qmp;   // p, q - p
  float2 half_q2;  // (q - 2) / 2
  float2 q2_l2;    // (q - 2) log2(1 / sigma)
};
__device__ __forceinline__ PriorK prior_k(const PriorC& c) {
  PriorK k;
  k.half_qp = f2(0.5f * c.qp);
  k.qp_l2 = f2(c.qp_l2_inv_csig);
  k.p = f2(c.p);
  k.qmp = f2(c.qp);
  k.half_q2 = f2(0.5f * (c.q - 2.0f));
  k.q2_l2 = f2((c.q - 2.0f) * c.l2_inv_sig);
  return k;
}

// One neighbour term of the qGGMRF potential for two voxels at once (the two lanes):
//   rho(d)  = |d/sigma|^q / (1 + u),  u = |d/(c sigma)|^(q-p),  r = 1 / (1 + u)
//   rho'(d) = d/sigma^2 |d/sigma|^(q-2) (q + p u) / (1 + u)^2
//           = d/sigma^2 |d/sigma|^(q-2) r (p + (q - p) r)
// g += sigma^2 rho'(d) and, when phi, ph += sigma^2 rho(d) (the caller folds 1/sigma^2 into
// the neighbour weight).  u comes from log2(d^2 + 1e-30), which stays finite at d = 0 (there
// r = 1 and both terms vanish).  Three special-function operations per lane (log2, exp2,
// reciprocal), four for q != 2.
template <bool Q2>
__device__ __forceinline__ void nbr2(float2 y, float2 nb, const PriorK& k, float2& g, float2& ph, bool phi) {
  const float2 d = f2fma(nb, f2(-1.f), y);
  const float2 sq = f2fma(d, d, f2(1e-30f));
  const float2 la = make_float2(lg2a(sq.x), lg2a(sq.y));
  const float2 s = f2fma(k.half_qp, la, k.qp_l2);
  const float2 e = f2add(make_float2(ex2a(s.x), ex2a(s.y)), f2(1.f));
  const float2 r = make_float2(rcpa(e.x), rcpa(e.y));
  const float2 t = f2fma(k.qmp, r, k.p);
  float2 dr = f2mul(d, r);
  if constexpr (!Q2) {
    const float2 s2 = f2fma(k.half_q2, la, k.q2_l2);
    dr = f2mul(dr, make_float2(ex2a(s2.x), ex2a(s2.y)));
  }
  g = f2fma(dr, t, g);
  if (phi) ph = f2fma(d, dr, ph);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction of kParts values to partials[block]: fixed order, FP64.
template <int W>
__device__ __forceinline__ void block_partials(double (&acc)[kParts], double* red, double* out) {
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kParts; ++j) {
    double v = warp_sum(acc[j]);
    if (lane == 0) red[warp * kParts + j] = v;
  }
  __syncthreads();
  if (threadIdx.x < kParts) {
    double s = 0.0;
    for (int w = 0; w < W; ++w) s += red[w * kParts + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------- pass 1: rows, forward
template <int N, bool BF>
__global__ void __launch_bounds__(Geo<N>::THREADS) k_pass1(GroupDev g, StepArgs a) {
  using Gm = Geo<N>;
  using F = typename Gm::F;
  constexpr int T = Gm::T, P = Gm::P, G = Gm::G, RB = Gm::RB, LD = Gm::LD;
  extern __shared__ float2 sm[];
  const float *x, *xp;
  float beta;
  if (a.st) {
    if (skip_iter<BF>(a.st)) return;
    int cur = a.st->cur;
    x = a.xb[cur];
    xp = a.xb[(cur + 2) % 3];
    beta = (float)a.st->beta;
  } else {
    x = a.x;
    xp = a.xprev;
    beta = a.beta;
  }
  const int s = blockIdx.x / Gm::NB, rb = blockIdx.x % Gm::NB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / T, t = lane % T;
  const int rl = warp * G + grp;
  const int r = rb * RB + rl;
  const size_t base = g.img_off + ((size_t)s * N + r) * N;

  // packed real row: z[n] = y[2n] + i y[2n+1], nonzero for n < N/2 (the rest is padding)
  float2 v[P];
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    if constexpr (i < P / 2) {
      const int n = t + T * i;
      float2 xv = __ldg(reinterpret_cast<const float2*>(x + base) + n);
      float2 pv = __ldg(reinterpret_cast<const float2*>(xp + base) + n);
      v[i] = make_float2(fmaf(beta, xv.x - pv.x, xv.x), fmaf(beta, xv.y - pv.y, xv.y));
    } else {
      v[i] = make_float2(0.f, 0.f);
    }
  });
  F::template run<-1>(v, sm + (warp * G + grp) * F::SMEM, g.twN, t);

  // split the packed transform: Y[v] = E[v] + w^v O[v], needs Z[v] and Z[N - v]
  float2 y[P];
  const int partner = (T - t) % T;
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    float2 zo = v[P - 1 - i];
    float2 zs;
    zs.x = __shfl_sync(0xffffffffu, zo.x, partner, T);
    zs.y = __shfl_sync(0xffffffffu, zo.y, partner, T);
    if (t == 0) zs = v[(P - i) % P];
    float2 z = v[i];
    float2 e = make_float2(0.5f * (z.x + zs.x), 0.5f * (z.y - zs.y));
    float2 o = make_float2(0.5f * (z.y + zs.y), -0.5f * (z.x - zs.x));
    float2 w = __ldg(&g.twM[t + T * i]);
    y[i] = cadd(e, cmul(w, o));
  });
  const float nyq = v[0].x - v[0].y;
  __syncthreads();
  float2* tb = sm;
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    tb[rl * LD + t + T * i] = y[i];
  });
  if (t == 0) tb[rl * LD + N] = make_float2(nyq, 0.f);
  __syncthreads();
  using IO = SpecIO<BF>;
  typename IO::T* out = reinterpret_cast<typename IO::T*>(g.spec) + (size_t)s * (N + 1) * N + rb * RB;
  for (int e = threadIdx.x; e < (N + 1) * RB; e += Gm::THREADS) {
    const int vv = e / RB, rr = e - vv * RB;
    IO::st(out, (size_t)vv * N + rr, tb[rr * LD + vv]);
  }
}

// ---------------------------------------------------------------- pass 2: columns
template <int N, bool BF>
__global__ void __launch_bounds__(Geo<N>::THREADS) k_pass2(GroupDev g, const IterState* st) {
  using Gm = Geo<N>;
  using F = typename Gm::F;
  constexpr int T = Gm::T, P = Gm::P, G = Gm::G;
  extern __shared__ float2 sm[];
  if (st && skip_iter<BF>(st)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / T, t = lane % T;
  const int unit = warp * G + grp, h = unit & 1;
  const int col = blockIdx.x * Gm::CPB + (unit >> 1);
  const int ncols = g.S * (N + 1);
  const bool active = col < ncols;
  const int vcol = active ? col / g.S : 0, s = active ? col % g.S : 0;  // slices fastest: kernel column reuse
  using IO = SpecIO<BF>;
  typename IO::T* p = reinterpret_cast<typename IO::T*>(g.spec) + ((size_t)s * (N + 1) + vcol) * N;
  float2 v[P];
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const int rr = t + T * i;
    float2 w = active ? IO::ld(p, rr) : make_float2(0.f, 0.f);
    if (h) w = cmul(w, __ldg(&g.twM[rr]));  // odd half: w[r] * exp(-2 pi i r / 2N)
    v[i] = w;
  });
  float2* xs = sm + unit * F::SMEM;
  F::template run<-1>(v, xs, g.twN, t);
  const float* cc = g.chat + ((size_t)vcol * 2 + h) * N;
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const float c = __ldg(&cc[t + T * i]);
    v[i] = make_float2(v[i].x * c, v[i].y * c);
  });
  F::template run<1>(v, xs, g.twN, t);
  if (h) {
    SFor<0, P>::run([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      v[i] = cmulc(v[i], __ldg(&g.twM[t + T * i]));
    });
  }
  // even and odd units can share a warp (N <= 512): every lane reaches this barrier
  __syncwarp();
  if (h) {
    SFor<0, P>::run([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      xs[t + T * i] = v[i];
    });
  }
  __syncthreads();
  if (!h && active) {
    const float2* os = sm + (unit + 1) * F::SMEM;
    SFor<0, P>::run([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      const int rr = t + T * i;
      IO::st(p, rr, cadd(v[i], os[rr]));
    });
  }
}

// ---------------------------------------------------------------- pass 3a: rows, inverse
// Inverse packed real row transform of every row (one row group per warp, RB rows per block,
// the layout of pass 1), crop to the first N columns: K (*) y written row-major as FP32.
template <int N, bool BF>
__global__ void __launch_bounds__(Geo<N>::THREADS) k_pass3a(GroupDev g, const IterState* st, float* kz) {
  using Gm = Geo<N>;
  using F = typename Gm::F;
  constexpr int T = Gm::T, P = Gm::P, G = Gm::G, RB = Gm::RB, LD = Gm::LD;
  extern __shared__ float2 sm[];
  if (st && skip_iter<BF>(st)) return;
  const int s = blockIdx.x / Gm::NB, rb = blockIdx.x % Gm::NB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / T, t = lane % T;
  const int rl = warp * G + grp;
  const int r0 = rb * RB;
  float2* tb = sm;
  {
    using IO = SpecIO<BF>;
    const typename IO::T* sp = reinterpret_cast<const typename IO::T*>(g.spec) + (size_t)s * (N + 1) * N + r0;
    for (int e = threadIdx.x; e < (N + 1) * RB; e += Gm::THREADS) {
      const int vv = e / RB, rr = e - vv * RB;
      tb[rr * LD + vv] = IO::ld(sp, (size_t)vv * N + rr);
    }
  }
  __syncthreads();
  // the length-2N real inverse as a length-N complex inverse of Z[v] = E[v] + i O[v]
  float2 q[P];
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const int vp = t + T * i;
    const float2 zv = tb[rl * LD + vp];
    const float2 zr = tb[rl * LD + N - vp];
    const float2 e = make_float2(zv.x + zr.x, zv.y - zr.y);
    const float2 d = make_float2(zv.x - zr.x, zv.y + zr.y);
    const float2 o = cmulc(d, __ldg(&g.twM[vp]));
    q[i] = make_float2(e.x - o.y, e.y + o.x);
  });
  __syncthreads();
  F::template run<1>(q, sm + (warp * G + grp) * F::SMEM, g.twN, t);
  // the first N/2 packed outputs are the N kept columns
  float2* out = reinterpret_cast<float2*>(kz + ((size_t)s * N + r0 + rl) * N);
  SFor<0, P / 2>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    out[t + T * i] = q[i];
  });
}

// ---------------------------------------------------------------- passes 1, 2, 3a for 1536 and 2560
// The same three passes with block-wide FFTs (block_fft.cuh) instead of group FFTs: a block of
// 256 threads transforms one row or column at a time.  Layouts, scaling and the packed-real
// split are those of the group-FFT passes.
template <int N>
struct BGeo {
  static constexpr int THREADS = 256;
  static constexpr int RB = Geo<N>::RB;             // rows per block, as the stencil expects
  static constexpr int NB = N / RB;
  static constexpr int LD = N + 4;
  static constexpr size_t SM_ROWS = (size_t)(2 * N + RB * LD) * sizeof(float2);  // X, Y, RB staged rows
  static constexpr size_t SM_COL = (size_t)4 * N * sizeof(float2);              // X, Y, column, sum
};

template <int N, bool BF>
__global__ void __launch_bounds__(256) k_pass1_b(GroupDev g, StepArgs a) {
  using BG = BGeo<N>;
  extern __shared__ float2 sm[];
  const float *x, *xp;
  float beta;
  if (a.st) {
    if (skip_iter<BF>(a.st)) return;
    const int cur = a.st->cur;
    x = a.xb[cur];
    xp = a.xb[(cur + 2) % 3];
    beta = (float)a.st->beta;
  } else {
    x = a.x;
    xp = a.xprev;
    beta = a.beta;
  }
  const int s = blockIdx.x / BG::NB, rb = blockIdx.x % BG::NB;
  float2* X = sm;
  float2* Y = sm + N;
  float2* tb = sm + 2 * N;
  for (int rr = 0; rr < BG::RB; ++rr) {
    __syncthreads();  // the previous row's transform has been read
    const size_t base = g.img_off + ((size_t)s * N + rb * BG::RB + rr) * N;
    // packed real row z[n] = y[2n] + i y[2n+1] for n < N/2, zero padding above
    for (int n = threadIdx.x; n < N; n += BG::THREADS) {
      float2 v = make_float2(0.f, 0.f);
      if (n < N / 2) {
        const float2 xv = __ldg(reinterpret_cast<const float2*>(x + base) + n);
        const float2 pv = __ldg(reinterpret_cast<const float2*>(xp + base) + n);
        v = make_float2(fmaf(beta, xv.x - pv.x, xv.x), fmaf(beta, xv.y - pv.y, xv.y));
      }
      X[n] = v;
    }
    const float2* Z = block_fft<N, -1>(X, Y, g.twN);
    // Y[v] = E[v] + w^v O[v] from Z[v] and Z[N - v]; the Nyquist term Y[N] = Re Z0 - Im Z0
    for (int v = threadIdx.x; v < N; v += BG::THREADS) {
      const float2 z = Z[v], zs = Z[(N - v) % N];
      const float2 e = make_float2(0.5f * (z.x + zs.x), 0.5f * (z.y - zs.y));
      const float2 o = make_float2(0.5f * (z.y + zs.y), -0.5f * (z.x - zs.x));
      tb[rr * BG::LD + v] = cadd(e, cmul(__ldg(&g.twM[v]), o));
    }
    if (threadIdx.x == 0) tb[rr * BG::LD + N] = make_float2(Z[0].x - Z[0].y, 0.f);
  }
  __syncthreads();
  using IO = SpecIO<BF>;
  typename IO::T* out = reinterpret_cast<typename IO::T*>(g.spec) + (size_t)s * (N + 1) * N + rb * BG::RB;
  for (int e = threadIdx.x; e < (N + 1) * BG::RB; e += BG::THREADS) {
    const int vv = e / BG::RB, rr = e - vv * BG::RB;
    IO::st(out, (size_t)vv * N + rr, tb[rr * BG::LD + vv]);
  }
}

template <int N, bool BF>
__global__ void __launch_bounds__(256) k_pass2_b(GroupDev g, const IterState* st) {
  using BG = BGeo<N>;
  extern __shared__ float2 sm[];
  if (st && skip_iter<BF>(st)) return;
  const int vcol = blockIdx.x / g.S, s = blockIdx.x % g.S;  // slices fastest: kernel column reuse
  using IO = SpecIO<BF>;
  typename IO::T* p = reinterpret_cast<typename IO::T*>(g.spec) + ((size_t)s * (N + 1) + vcol) * N;
  float2* X = sm;
  float2* Y = sm + N;
  float2* col = sm + 2 * N;
  float2* sum = sm + 3 * N;
  for (int r = threadIdx.x; r < N; r += BG::THREADS) col[r] = IO::ld(p, r);
  for (int h = 0; h < 2; ++h) {
    __syncthreads();
    // even half: the column; odd half: the column times exp(-2 pi i r / 2N)
    for (int r = threadIdx.x; r < N; r += BG::THREADS) X[r] = h ? cmul(col[r], __ldg(&g.twM[r])) : col[r];
    float2* F = block_fft<N, -1>(X, Y, g.twN);
    const float* cc = g.chat + ((size_t)vcol * 2 + h) * N;
    for (int k = threadIdx.x; k < N; k += BG::THREADS) {
      const float c = __ldg(&cc[k]);
      F[k] = make_float2(F[k].x * c, F[k].y * c);
    }
    float2* G = block_fft<N, 1>(F, F == X ? Y : X, g.twN);
    for (int r = threadIdx.x; r < N; r += BG::THREADS) {
      const float2 v = h ? cmulc(G[r], __ldg(&g.twM[r])) : G[r];
      sum[r] = h ? cadd(sum[r], v) : v;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < N; r += BG::THREADS) IO::st(p, r, sum[r]);
}

template <int N, bool BF>
__global__ void __launch_bounds__(256) k_pass3a_b(GroupDev g, const IterState* st, float* kz) {
  using BG = BGeo<N>;
  extern __shared__ float2 sm[];
  if (st && skip_iter<BF>(st)) return;
  const int s = blockIdx.x / BG::NB, rb = blockIdx.x % BG::NB;
  const int r0 = rb * BG::RB;
  float2* X = sm;
  float2* Y = sm + N;
  float2* tb = sm + 2 * N;
  {
    using IO = SpecIO<BF>;
    const typename IO::T* sp = reinterpret_cast<const typename IO::T*>(g.spec) + (size_t)s * (N + 1) * N + r0;
    for (int e = threadIdx.x; e < (N + 1) * BG::RB; e += BG::THREADS) {
      const int vv = e / BG::RB, rr = e - vv * BG::RB;
      tb[rr * BG::LD + vv] = IO::ld(sp, (size_t)vv * N + rr);
    }
  }
  for (int rr = 0; rr < BG::RB; ++rr) {
    __syncthreads();
    // the length-2N real inverse as a length-N complex inverse of Z[v] = E[v] + i O[v]
    for (int vp = threadIdx.x; vp < N; vp += BG::THREADS) {
      const float2 zv = tb[rr * BG::LD + vp];
      const float2 zr = tb[rr * BG::LD + N - vp];
      const float2 e = make_float2(zv.x + zr.x, zv.y - zr.y);
      const float2 d = make_float2(zv.x - zr.x, zv.y + zr.y);
      const float2 o = cmulc(d, __ldg(&g.twM[vp]));
      X[vp] = make_float2(e.x - o.y, e.y + o.x);
    }
    const float2* Z = block_fft<N, 1>(X, Y, g.twN);
    float2* out = reinterpret_cast<float2*>(kz + ((size_t)s * N + r0 + rr) * N);
    for (int n = threadIdx.x; n < N / 2; n += BG::THREADS) out[n] = Z[n];
  }
}

// ---------------------------------------------------------------- pass 3b: gradient and update
// A block owns RB consecutive rows of one group and marches through a chunk of its slices,
// keeping y for slices z-1, z, z+1 (rows -1 .. RB) in a three-slot ring so every slice of y is
// read from memory once per chunk.  Per slice each thread walks its voxels and sums rho' over
// the 26 neighbours.  The voxel loop is a plain runtime loop so the unrolled neighbourhood
// stays small enough for the instruction cache.  Each unordered neighbour pair enters Phi
// once, from the voxel it is a forward offset of.  With only the ring in shared memory and no
// transform registers, three blocks of eight warps fit an SM (one at N = 2048).
template <int N>
struct Geo3 {
  using Gm = Geo<N>;
  static constexpr int RB = Gm::RB, W = 2 * Gm::W, THREADS = 32 * W;
  static constexpr int ROWS = RB + 2;  // ring rows (one halo row each side)
  static constexpr size_t SM = (size_t)3 * ROWS * N * sizeof(float);
  static constexpr int MINB = SM * 3 <= 220 * 1024 ? 3 : 1;
};

// y = x + beta (x - x_prev) for block rows -1 .. RB of one slice into a ring slot (zero outside)
template <int N>
__device__ __forceinline__ void load_ring(float* slot, const float* x, const float* xp, float beta, size_t off_slice,
                                          int r0) {
  using G3 = Geo3<N>;
  for (int e = threadIdx.x; e < G3::ROWS * (N / 4); e += G3::THREADS) {
    const int c4 = e % (N / 4), rowi = e / (N / 4);
    const int rr = r0 - 1 + rowi;
    float4 yv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (rr >= 0 && rr < N) {
      const size_t off = off_slice + (size_t)rr * N;
      const float4 xv = __ldg(reinterpret_cast<const float4*>(x + off) + c4);
      const float4 pv = __ldg(reinterpret_cast<const float4*>(xp + off) + c4);
      yv = make_float4(fmaf(beta, xv.x - pv.x, xv.x), fmaf(beta, xv.y - pv.y, xv.y), fmaf(beta, xv.z - pv.z, xv.z),
                       fmaf(beta, xv.w - pv.w, xv.w));
    }
    reinterpret_cast<float4*>(slot + rowi * N)[c4] = yv;
  }
}

// kz: K (*) y of the group from pass 3a ([slice][row][col]); phase: in Iterate mode, the storage
// phase this launch belongs to (0 FP32, 1 BF16), checked like the other passes.
template <int N, int MODE, bool Q2>
__global__ void __launch_bounds__(Geo3<N>::THREADS, Geo3<N>::MINB)
    k_pass3(GroupDev g, StepArgs a, PriorC pc, const float* __restrict__ kz, int phase, double* partials,
            int block_offset, int zc) {
  using Gm = Geo<N>;
  using G3 = Geo3<N>;
  constexpr int RB = Gm::RB, ROWS = G3::ROWS;
  constexpr bool PRIOR = MODE != (int)Pass3Mode::Apply;
  constexpr bool PHI = MODE == (int)Pass3Mode::Step || MODE == (int)Pass3Mode::Iterate ||
                       MODE == (int)Pass3Mode::Objective;
  constexpr bool UPDATE = MODE == (int)Pass3Mode::Step || MODE == (int)Pass3Mode::Iterate;
  extern __shared__ float2 sm[];
  __shared__ double red[G3::W * kParts];
  const float *x, *xp;
  float* out;
  float beta, invL;
  if constexpr (MODE == (int)Pass3Mode::Iterate) {
    if (a.st->done || a.st->bf16 != phase) return;
    const int cur = a.st->cur;
    x = cur == 0 ? a.xb[0] : (cur == 1 ? a.xb[1] : a.xb[2]);
    xp = cur == 0 ? a.xb[2] : (cur == 1 ? a.xb[0] : a.xb[1]);
    out = cur == 0 ? a.xb[1] : (cur == 1 ? a.xb[2] : a.xb[0]);
    beta = (float)a.st->beta;
    invL = (float)a.st->invL;
  } else {
    x = a.x;
    xp = a.xprev;
    out = a.out;
    beta = a.beta;
    invL = a.invL;
  }
  const int rb = blockIdx.x % Gm::NB, chunk = blockIdx.x / Gm::NB;
  const int z0 = chunk * zc, z1 = min(g.S, z0 + zc);
  const int r0 = rb * RB;
  float* ring = reinterpret_cast<float*>(sm);
  const size_t N2 = (size_t)N * N;
  // neighbour weights with 1/sigma^2 folded in: nbr2 sums sigma^2 rho' and sigma^2 rho
  const float2 wf = f2(pc.wf * pc.inv_sig2), we = f2(pc.we * pc.inv_sig2), wc = f2(pc.wc * pc.inv_sig2);
  const float2 lam = f2(pc.lam);
  const PriorK pk = prior_k(pc);
  constexpr int H = N / 2;
  static_assert(H % 32 == 0, "a warp must cover one row segment");

  double dacc[kParts];
#pragma unroll
  for (int j = 0; j < kParts; ++j) dacc[j] = 0.0;

  if constexpr (PRIOR) {
    load_ring<N>(ring + (z0 % 3) * ROWS * N, x, xp, beta, g.img_off + (size_t)z0 * N2, r0);
    if (z0 > 0) load_ring<N>(ring + ((z0 + 2) % 3) * ROWS * N, x, xp, beta, g.img_off + (size_t)(z0 - 1) * N2, r0);
  }

  for (int z = z0; z < z1; ++z) {
    const size_t slice_base = g.img_off + (size_t)z * N2;
    // the ring slot of slice z+1 is free once every thread has finished slice z-1
    if constexpr (PRIOR) {
      __syncthreads();
      if (z + 1 < g.S) load_ring<N>(ring + ((z + 1) % 3) * ROWS * N, x, xp, beta, slice_base + N2, r0);
      __syncthreads();
    }
    const float* kzr = kz + (size_t)z * N2 + (size_t)r0 * N;

    // ---- per voxel: prior, gradient, update, partial sums.  A thread takes the voxels in
    // columns c and c + N/2 of one block row as the two lanes of packed FP32 pairs (a warp
    // covers 32 consecutive c of one row, so the row and slice tests are warp-uniform).
    const float* sz[3] = {ring + ((z + 2) % 3) * ROWS * N, ring + (z % 3) * ROWS * N, ring + ((z + 1) % 3) * ROWS * N};
    const bool zval0 = z > 0, zval2 = z + 1 < g.S;
    float2 acc[kParts];
#pragma unroll
    for (int j = 0; j < kParts; ++j) acc[j] = f2(0.f);
#pragma unroll 1
    for (int i = threadIdx.x; i < RB * H; i += G3::THREADS) {
      const int row = i / H, c = i - row * H;
      const int grow = r0 + row;
      const size_t ia = slice_base + (size_t)grow * N + c, ib = ia + H;
      const float2 zd = make_float2(__ldg(kzr + row * N + c), __ldg(kzr + row * N + c + H));
      if constexpr (!PRIOR) {
        // Apply: pass 3a wrote K (*) x to the output itself; only the partial sums remain
        const float2 xv = make_float2(__ldg(x + ia), __ldg(x + ib));
        acc[0] = f2fma(xv, zd, acc[0]);
        acc[5] = f2fma(zd, zd, acc[5]);
      } else {
        const float2 at = make_float2(__ldg(a.atg + ia), __ldg(a.atg + ib));
        float2 xv = f2(0.f);
        if constexpr (UPDATE) xv = make_float2(__ldg(x + ia), __ldg(x + ib));
        const float* ry = sz[1] + (row + 1) * N;
        const float2 yv = make_float2(ry[c], ry[c + H]);
        // missing neighbours (free boundary) read the voxel itself: d = 0 adds nothing
        const bool hasL = c > 0, hasR = c + 1 < H;  // column 0 (lane x), column N - 1 (lane y)
        const int cl = hasL ? c - 1 : c, cr = hasR ? c + H + 1 : c + H;
        float2 gp[3], ph[3];  // by neighbour class: face, edge, corner
#pragma unroll
        for (int j = 0; j < 3; ++j) gp[j] = ph[j] = f2(0.f);
#pragma unroll
        for (int dz = 0; dz < 3; ++dz) {
          if ((dz == 0 && !zval0) || (dz == 2 && !zval2)) continue;
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) {
            if ((dy == 0 && grow == 0) || (dy == 2 && grow + 1 == N)) continue;
            const float* rp = sz[dz] + (row + dy) * N;
            const int cls = (dz != 1) + (dy != 1);  // class of the dx = -1, +1 neighbours
            const bool fwd = dz > 1 || (dz == 1 && dy > 1);
            const float2 nbL = make_float2(hasL ? rp[cl] : yv.x, rp[c + H - 1]);
            const float2 nbR = make_float2(rp[c + 1], hasR ? rp[cr] : yv.y);
            if (cls > 0) nbr2<Q2>(yv, make_float2(rp[c], rp[c + H]), pk, gp[cls - 1], ph[cls - 1], PHI && fwd);
            nbr2<Q2>(yv, nbL, pk, gp[cls], ph[cls], PHI && fwd);
            nbr2<Q2>(yv, nbR, pk, gp[cls], ph[cls], PHI && (fwd || cls == 0));
          }
        }
        const float2 gpv = f2fma(wc, gp[2], f2fma(we, gp[1], f2mul(wf, gp[0])));
        const float2 Gv = f2fma(lam, gpv, f2fma(at, f2(-1.f), zd));
        acc[0] = f2fma(yv, zd, acc[0]);
        acc[1] = f2fma(yv, at, acc[1]);
        if constexpr (PHI) acc[2] = f2add(acc[2], f2fma(wc, ph[2], f2fma(we, ph[1], f2mul(wf, ph[0]))));
        acc[4] = f2fma(Gv, Gv, acc[4]);
        if constexpr (MODE == (int)Pass3Mode::Gradient) {
          out[ia] = Gv.x;
          out[ib] = Gv.y;
        } else if constexpr (UPDATE) {
          const float2 xn = f2fma(f2(-invL), Gv, yv);
          out[ia] = xn.x;
          out[ib] = xn.y;
          acc[3] = f2fma(Gv, f2fma(xv, f2(-1.f), xn), acc[3]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kParts; ++j) dacc[j] += (double)acc[j].x + (double)acc[j].y;
  }
  block_partials<G3::W>(dacc, red, partials + (size_t)(block_offset + blockIdx.x) * kParts);
}

// ---------------------------------------------------------------- host launchers
template <int N>
static int set_smem_limits() {
  using Gm = Geo<N>;
  static bool done = false;
  if (done) return TMBIR_OK;
  if constexpr (is_block_fft_size<N>()) {
    using BG = BGeo<N>;
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass1_b<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BG::SM_ROWS));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass1_b<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BG::SM_ROWS));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass2_b<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BG::SM_COL));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass2_b<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BG::SM_COL));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass3a_b<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BG::SM_ROWS));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass3a_b<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BG::SM_ROWS));
  } else {
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass1<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::SM1));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass1<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::SM1));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass2<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::SM2));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass2<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::SM2));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass3a<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::SM1));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass3a<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::SM1));
  }
#define TMBIR_P3ATTR(M, Q)                                                                           \
  TMBIR_CUDA(cudaFuncSetAttribute(k_pass3<N, M, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)Geo3<N>::SM));
  TMBIR_P3ATTR(0, true) TMBIR_P3ATTR(1, true) TMBIR_P3ATTR(2, true) TMBIR_P3ATTR(3, true) TMBIR_P3ATTR(4, true)
  TMBIR_P3ATTR(1, false) TMBIR_P3ATTR(2, false) TMBIR_P3ATTR(3, false) TMBIR_P3ATTR(4, false)
#undef TMBIR_P3ATTR
  done = true;
  return TMBIR_OK;
}

template <int N>
static int pass1_n(const GroupDev& g, const StepArgs& a, bool bf16, cudaStream_t s) {
  using Gm = Geo<N>;
  if (int e = set_smem_limits<N>()) return e;
  if constexpr (is_block_fft_size<N>()) {
    using BG = BGeo<N>;
    if (bf16)
      k_pass1_b<N, true><<<g.S * BG::NB, BG::THREADS, BG::SM_ROWS, s>>>(g, a);
    else
      k_pass1_b<N, false><<<g.S * BG::NB, BG::THREADS, BG::SM_ROWS, s>>>(g, a);
  } else {
    if (bf16)
      k_pass1<N, true><<<g.S * Gm::NB, Gm::THREADS, Gm::SM1, s>>>(g, a);
    else
      k_pass1<N, false><<<g.S * Gm::NB, Gm::THREADS, Gm::SM1, s>>>(g, a);
  }
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
template <int N>
static int pass2_n(const GroupDev& g, const IterState* st, bool bf16, cudaStream_t s) {
  using Gm = Geo<N>;
  if (int e = set_smem_limits<N>()) return e;
  if constexpr (is_block_fft_size<N>()) {
    using BG = BGeo<N>;
    const int blocks = g.S * (N + 1);
    if (bf16)
      k_pass2_b<N, true><<<blocks, BG::THREADS, BG::SM_COL, s>>>(g, st);
    else
      k_pass2_b<N, false><<<blocks, BG::THREADS, BG::SM_COL, s>>>(g, st);
  } else {
    const int blocks = (g.S * (N + 1) + Gm::CPB - 1) / Gm::CPB;
    if (bf16)
      k_pass2<N, true><<<blocks, Gm::THREADS, Gm::SM2, s>>>(g, st);
    else
      k_pass2<N, false><<<blocks, Gm::THREADS, Gm::SM2, s>>>(g, st);
  }
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
template <int N, int MODE>
static int pass3_nm(const GroupDev& g, const StepArgs& a, const PriorC& pc, const float* kz, int phase,
                    double* partials, int off, cudaStream_t s) {
  using Gm = Geo<N>;
  const int zc = pass3_zc(g, Gm::NB);
  const int blocks = Gm::NB * ((g.S + zc - 1) / zc);
  if (pc.q_is_2 || MODE == 0)
    k_pass3<N, MODE, true><<<blocks, Geo3<N>::THREADS, Geo3<N>::SM, s>>>(g, a, pc, kz, phase, partials, off, zc);
  else
    k_pass3<N, MODE, false><<<blocks, Geo3<N>::THREADS, Geo3<N>::SM, s>>>(g, a, pc, kz, phase, partials, off, zc);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
// part: 1 pass 3a only, 2 pass 3b only, 3 both
template <int N>
static int pass3_n(const GroupDev& g, const StepArgs& a, Pass3Mode m, const PriorC& pc, double* partials, int off,
                   bool bf16, int part, cudaStream_t s) {
  using Gm = Geo<N>;
  if (int e = set_smem_limits<N>()) return e;
  if (bf16 && m != Pass3Mode::Iterate) return set_error(TMBIR_ERR_ARG, "BF16 spectra are an iteration option only");
  // Apply writes K (*) x straight into the output; every other mode into the group's buffer
  float* kz = m == Pass3Mode::Apply ? a.out + g.img_off : g.kz;
  const IterState* st = m == Pass3Mode::Iterate ? a.st : nullptr;
  if (part & 1) {
    if constexpr (is_block_fft_size<N>()) {
      using BG = BGeo<N>;
      if (bf16)
        k_pass3a_b<N, true><<<g.S * BG::NB, BG::THREADS, BG::SM_ROWS, s>>>(g, st, kz);
      else
        k_pass3a_b<N, false><<<g.S * BG::NB, BG::THREADS, BG::SM_ROWS, s>>>(g, st, kz);
    } else {
      if (bf16)
        k_pass3a<N, true><<<g.S * Gm::NB, Gm::THREADS, Gm::SM1, s>>>(g, st, kz);
      else
        k_pass3a<N, false><<<g.S * Gm::NB, Gm::THREADS, Gm::SM1, s>>>(g, st, kz);
    }
    TMBIR_CHECK_LAUNCH();
  }
  if (!(part & 2)) return TMBIR_OK;
  const int phase = bf16 ? 1 : 0;
  switch (m) {
    case Pass3Mode::Apply: return pass3_nm<N, 0>(g, a, pc, kz, phase, partials, off, s);
    case Pass3Mode::Gradient: return pass3_nm<N, 1>(g, a, pc, kz, phase, partials, off, s);
    case Pass3Mode::Step: return pass3_nm<N, 2>(g, a, pc, kz, phase, partials, off, s);
    case Pass3Mode::Iterate: return pass3_nm<N, 3>(g, a, pc, kz, phase, partials, off, s);
    default: return pass3_nm<N, 4>(g, a, pc, kz, phase, partials, off, s);
  }
}

}  // namespace tmbir
