// The per-iteration hot path: R*R y as a zero-padded 2N x 2N FFT convolution with the
// point-spread kernel (Sec. 2.1, Eq. 9), fused with -R*g (Eq. 11), the qGGMRF prior
// gradient over the 26-neighbourhood (Eq. 5, Sec. 2.4) and the fast-gradient update with
// restart (Sec. 2, Eq. 6).
//
// Four launches per iteration, each over every slice of a group:
//   pass 1  rows:    y = x_k + beta (x_k - x_{k-1}); real FFT of length 2N of each row (the
//                    upper N entries are the zero padding), written column-major
//                    spec[v][r], v = 0..N (half spectrum), r = 0..N-1 (nonzero rows only).
//   pass 2  columns: per column v, FFT of length 2N of the N nonzero rows, multiply by the
//                    real kernel spectrum, inverse FFT, keep the first N rows (the crop).
//                    The length-2N transforms are split into their even and odd halves, two
//                    length-N transforms each, so the zero padding and the crop cost nothing.
//   pass 3a rows:    inverse real FFT of each row, keep the first N columns -> K (*) y.
//   pass 3b stencil: per voxel G = K(*)y - R*g + lambda grad Phi(y) (each neighbour pair of the
//                    26-neighbourhood evaluated once), x_{k+1} = y - G/L, and the partial sums
//                    the optimiser needs (compensated FP32 per thread, FP64 per block).
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
#include "tc05.cuh"

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

// Copies count elements, e = threadIdx.x + k * NT, from ld(e) to st(e, v) in batches of B whose
// loads are all issued before their stores, so that a thread keeps B global loads in flight
// instead of waiting out each load's latency before the next.
template <int NT, int B, class Ld, class St>
__device__ __forceinline__ void batched_copy(int count, Ld&& ld, St&& st) {
  for (int e0 = threadIdx.x; e0 < count; e0 += B * NT) {
    float2 v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int e = e0 + b * NT;
      v[b] = e < count ? ld(e) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int e = e0 + b * NT;
      if (e < count) st(e, v[b]);
    }
  }
}

// ---------------------------------------------------------------- launch geometry
template <int N, int Wp = 4>
struct Geo {
  using F = typename FFTShape<N>::type;
  static constexpr int T = F::T, P = F::P, G = 32 / T;
  static constexpr int W = Wp;          // warps per block
  static constexpr int THREADS = 32 * W;
  static constexpr int RB = W * G;      // rows per block in passes 1 and 3
  static constexpr int NB = N / RB;     // row blocks per slice
  static constexpr int LD = N + 4;      // row stride (complex) of the row-major staging buffer
  static constexpr int UNITS = W * G;   // (column, half) units per block in pass 2
  static constexpr int CPB = UNITS / 2; // columns per block in pass 2
  static constexpr size_t SM_FFT = (size_t)W * G * F::SMEM * sizeof(float2);
  static constexpr size_t SM_TB = (size_t)RB * LD * sizeof(float2);
  static constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
  static constexpr size_t SM1 = cmax(SM_FFT, SM_TB);
  static constexpr size_t SM2 = SM_FFT;
};

// Launch shapes of pass 3a and pass 2 at N = 1024, chosen by measurement on GB300 (64 slices,
// 256 angles; ms per launch):
//   pass 3a: eight warps per block gather 8-row (64-byte) segments of the column-major
//            spectrum instead of 4-row (32-byte) ones; with at most 128 registers (two blocks
//            per SM) 0.211 ms against 0.262 with four warps (0.252 with eight warps at the
//            compiler's register choice, 0.278 at three blocks per SM).  Eight warps do not
//            help pass 1 (0.234 against 0.230), which keeps four.
//   pass 2:  at most 170 registers (three blocks per SM), 0.401 ms against 0.407 (128
//            registers: 0.588, spills).
// The other image sides keep four warps and the compiler's register choice.
#if defined(TMBIR_N) && TMBIR_N == 1024
#define TMBIR_P3A_BOUNDS(T) __launch_bounds__(T, 2)
#define TMBIR_P2_BOUNDS(T) __launch_bounds__(T, 3)
#else
#define TMBIR_P3A_BOUNDS(T) __launch_bounds__(T)
#define TMBIR_P2_BOUNDS(T) __launch_bounds__(T)
#endif
template <int N>
constexpr int pass3a_warps() {
  return N == 1024 ? 8 : 4;
}
template <int N>
using Geo3a = Geo<N, pass3a_warps<N>()>;

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
__global__ void __launch_bounds__(Geo<N>::THREADS) k_pass1(const __grid_constant__ GroupSet gs, StepArgs a) {
  using Gm = Geo<N>;
  using F = typename Gm::F;
  constexpr int T = Gm::T, P = Gm::P, G = Gm::G, RB = Gm::RB, LD = Gm::LD;
  extern __shared__ float2 sm[];
  int bid_;
  const int gi_ = gs.pick(bid_);
  const GroupDev& g = gs.g[gi_];
  const float *x, *xp;
  float beta;
  if (a.st) {
    if (skip_iter<BF>(a.st)) return;
    int cur = a.st->cur;
    // selects rather than an indexed parameter array, which would be copied to local memory
    x = cur == 0 ? a.xb[0] : (cur == 1 ? a.xb[1] : a.xb[2]);
    xp = cur == 0 ? a.xb[2] : (cur == 1 ? a.xb[0] : a.xb[1]);
    beta = (float)(a.gm + gi_)->beta;
  } else {
    x = a.x;
    xp = a.xprev;
    beta = a.beta;
  }
  const int s = bid_ / Gm::NB, rb = bid_ % Gm::NB;
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
// Column order of pass 2: chunks of kColChunk slices, and within a chunk the slices fastest, so
// that consecutive blocks share a column of the kernel spectrum (L2 reuse) while the blocks in
// flight stay within a few hundred MB of the spectrum instead of spreading over every slice of
// a large volume (TLB reach).  Column index -> (kernel column vcol, slice s).
constexpr int kColChunk = 16;
__device__ __forceinline__ void column_of(int col, int S, int ncol, int& vcol, int& s) {
  const int chunk = col / (kColChunk * ncol);
  const int within = col - chunk * kColChunk * ncol;
  const int rem = min(kColChunk, S - chunk * kColChunk);
  vcol = within / rem;
  s = chunk * kColChunk + (within - vcol * rem);
}

template <int N, bool BF>
__global__ void TMBIR_P2_BOUNDS(Geo<N>::THREADS) k_pass2(const __grid_constant__ GroupSet gs, const IterState* st) {
  using Gm = Geo<N>;
  using F = typename Gm::F;
  constexpr int T = Gm::T, P = Gm::P, G = Gm::G;
  extern __shared__ float2 sm[];
  int bid_;
  const int gi_ = gs.pick(bid_);
  const GroupDev& g = gs.g[gi_];
  if (st && skip_iter<BF>(st)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / T, t = lane % T;
  const int unit = warp * G + grp, h = unit & 1;
  const int col = bid_ * Gm::CPB + (unit >> 1);
  const int ncols = g.S * (N + 1);
  const bool active = col < ncols;
  int vcol = 0, s = 0;
  if (active) column_of(col, g.S, N + 1, vcol, s);
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
__global__ void TMBIR_P3A_BOUNDS(Geo3a<N>::THREADS) k_pass3a(const __grid_constant__ GroupSet gs, const IterState* st, float* apply_out) {
  using Gm = Geo3a<N>;
  using F = typename Gm::F;
  constexpr int T = Gm::T, P = Gm::P, G = Gm::G, RB = Gm::RB, LD = Gm::LD;
  extern __shared__ float2 sm[];
  int bid_;
  const int gi_ = gs.pick(bid_);
  const GroupDev& g = gs.g[gi_];
  float* kz = apply_out ? apply_out + g.img_off : g.kz;
  if (st && skip_iter<BF>(st)) return;
  const int s = bid_ / Gm::NB, rb = bid_ % Gm::NB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / T, t = lane % T;
  const int rl = warp * G + grp;
  const int r0 = rb * RB;
  float2* tb = sm;
  {
    using IO = SpecIO<BF>;
    const typename IO::T* sp = reinterpret_cast<const typename IO::T*>(g.spec) + (size_t)s * (N + 1) * N + r0;
    if constexpr (!BF) {
      // RB-row segments of the column-major spectrum, gathered by asynchronous 8-byte copies so
      // that every thread has all of its loads in flight at once
      for (int e = threadIdx.x; e < (N + 1) * RB; e += Gm::THREADS) {
        const int vv = e / RB, rr = e - vv * RB;
        tc05::cp_async8(&tb[rr * LD + vv], sp + (size_t)vv * N + rr);
      }
      tc05::cp_async_wait_all();
    } else {
      batched_copy<Gm::THREADS, 8>(
          (N + 1) * RB, [&](int e) { return IO::ld(sp, (size_t)(e / RB) * N + e % RB); },
          [&](int e, float2 v) { tb[(e % RB) * LD + e / RB] = v; });
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
__global__ void __launch_bounds__(256) k_pass1_b(const __grid_constant__ GroupSet gs, StepArgs a) {
  using BG = BGeo<N>;
  extern __shared__ float2 sm[];
  int bid_;
  const int gi_ = gs.pick(bid_);
  const GroupDev& g = gs.g[gi_];
  const float *x, *xp;
  float beta;
  if (a.st) {
    if (skip_iter<BF>(a.st)) return;
    const int cur = a.st->cur;
    // selects rather than an indexed parameter array, which would be copied to local memory
    x = cur == 0 ? a.xb[0] : (cur == 1 ? a.xb[1] : a.xb[2]);
    xp = cur == 0 ? a.xb[2] : (cur == 1 ? a.xb[0] : a.xb[1]);
    beta = (float)(a.gm + gi_)->beta;
  } else {
    x = a.x;
    xp = a.xprev;
    beta = a.beta;
  }
  const int s = bid_ / BG::NB, rb = bid_ % BG::NB;
  float2* X = sm;
  float2* Y = sm + N;
  float2* tb = sm + 2 * N;
  for (int rr = 0; rr < BG::RB; ++rr) {
    __syncthreads();  // the previous row's transform has been read
    const size_t base = g.img_off + ((size_t)s * N + rb * BG::RB + rr) * N;
    // packed real row z[n] = y[2n] + i y[2n+1] for n < N/2, zero padding above
    batched_copy<BG::THREADS, 4>(
        N / 2,
        [&](int n) {
          const float2 xv = __ldg(reinterpret_cast<const float2*>(x + base) + n);
          const float2 pv = __ldg(reinterpret_cast<const float2*>(xp + base) + n);
          return make_float2(fmaf(beta, xv.x - pv.x, xv.x), fmaf(beta, xv.y - pv.y, xv.y));
        },
        [&](int n, float2 v) { X[n] = v; });
    for (int n = N / 2 + threadIdx.x; n < N; n += BG::THREADS) X[n] = make_float2(0.f, 0.f);
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
__global__ void __launch_bounds__(256) k_pass2_b(const __grid_constant__ GroupSet gs, const IterState* st) {
  using BG = BGeo<N>;
  extern __shared__ float2 sm[];
  int bid_;
  const int gi_ = gs.pick(bid_);
  const GroupDev& g = gs.g[gi_];
  if (st && skip_iter<BF>(st)) return;
  int vcol, s;
  column_of(bid_, g.S, N + 1, vcol, s);
  using IO = SpecIO<BF>;
  typename IO::T* p = reinterpret_cast<typename IO::T*>(g.spec) + ((size_t)s * (N + 1) + vcol) * N;
  float2* X = sm;
  float2* Y = sm + N;
  float2* col = sm + 2 * N;
  float2* sum = sm + 3 * N;
  batched_copy<BG::THREADS, 8>(N, [&](int r) { return IO::ld(p, r); }, [&](int r, float2 v) { col[r] = v; });
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
__global__ void __launch_bounds__(256) k_pass3a_b(const __grid_constant__ GroupSet gs, const IterState* st, float* apply_out) {
  using BG = BGeo<N>;
  extern __shared__ float2 sm[];
  int bid_;
  const int gi_ = gs.pick(bid_);
  const GroupDev& g = gs.g[gi_];
  float* kz = apply_out ? apply_out + g.img_off : g.kz;
  if (st && skip_iter<BF>(st)) return;
  const int s = bid_ / BG::NB, rb = bid_ % BG::NB;
  const int r0 = rb * BG::RB;
  float2* X = sm;
  float2* Y = sm + N;
  float2* tb = sm + 2 * N;
  {
    using IO = SpecIO<BF>;
    const typename IO::T* sp = reinterpret_cast<const typename IO::T*>(g.spec) + (size_t)s * (N + 1) * N + r0;
    batched_copy<BG::THREADS, 8>(
        (N + 1) * BG::RB, [&](int e) { return IO::ld(sp, (size_t)(e / BG::RB) * N + e % BG::RB); },
        [&](int e, float2 v) { tb[(e % BG::RB) * BG::LD + e / BG::RB] = v; });
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

// ---------------------------------------------------------------- passes 1, 2, 3a for N = 2048
// At N = 2048 a thread of the register group FFT would hold 64 complex values (254 registers,
// spills in pass 2).  The zero padding lets each transform split into transforms of half the
// length, so these passes run the 1024-point group FFT of N = 1024 (32 threads x 32 values),
// one warp per part, with the same layouts and scaling as the group-FFT passes
// (w = exp(-2 pi i / 2048), W = exp(-2 pi i / 4096)):
//   pass 1: the packed row z has 1024 nonzero values of 2048, so
//           Z[2k + j] = DFT_1024(z[m] w^(jm))[k], j = 0, 1 (two warps per row);
//   pass 2: the column c has 2048 nonzero values of 4096, so
//           X[4k + j] = DFT_1024(W^(jm) (c[m] + (-i)^j c[m + 1024]))[k], j = 0..3 (four warps
//           per column); after the kernel multiply the kept rows n = m + 1024 q are
//           sum_j W^(-jm) i^(jq) u_j[m], u_j the inverse 1024-point transforms;
//   pass 3a: only the first 1024 packed outputs are kept, z[n] = sum_j w^(-jn) u_j[n], u_j the
//           inverse 1024-point transforms of Z[2k + j], j = 0, 1 (two warps per row).
// Each has the flops of the unsplit transforms (the split is the first radix-2 or radix-4
// stage, pruned by the padding and the crop).
struct Q2048 {
  static constexpr int N = 2048, H = 1024;
  using F = GroupFFT<32, 32>;
  static constexpr int LDZ = N + 4;  // row stride (complex) of staged rows
  // rows per block of passes 1 and 3a (two warps per row): 4 or 8, chosen per group by the
  // autotuner (GroupDev::rb1, rb3); eight rows write and gather 64-byte segments of the
  // column-major spectrum but hold one 135 KB block per SM, four rows 32-byte segments with two
  // or three blocks per SM whose phases overlap
  static constexpr int RB1 = 4;      // default of pass 1
  static constexpr int RB3 = 8;      // default of pass 3a
  template <int RB>
  static constexpr size_t sm_rows() {  // staged rows and the warps' exchange buffers, aliased
    return (size_t)(RB * LDZ > 2 * RB * F::SMEM ? RB * LDZ : 2 * RB * F::SMEM) * sizeof(float2);
  }
  static constexpr size_t SM2 = (size_t)(N + 4 * F::SMEM) * sizeof(float2);  // column + 4 exchange buffers
};

// W^n = exp(-2 pi i n / 4096) for 0 <= n < 4096 from the table of n < 2048 (W^(n + 2048) = -W^n)
__device__ __forceinline__ float2 tw4096(const float2* __restrict__ twM, int n) {
  const float2 w = __ldg(&twM[n & 2047]);
  return n < 2048 ? w : make_float2(-w.x, -w.y);
}

template <bool BF, int RB>
__global__ void __launch_bounds__(64 * RB) k_pass1_q(const __grid_constant__ GroupSet gs, StepArgs a) {
  using Q = Q2048;
  constexpr int N = Q::N, T = 32, P = 32, LDZ = Q::LDZ, THREADS = 64 * RB, NB = N / RB;
  extern __shared__ float2 sm[];
  int bid_;
  const int gi_ = gs.pick(bid_);
  const GroupDev& g = gs.g[gi_];
  const float *x, *xp;
  float beta;
  if (a.st) {
    if (skip_iter<BF>(a.st)) return;
    const int cur = a.st->cur;
    x = cur == 0 ? a.xb[0] : (cur == 1 ? a.xb[1] : a.xb[2]);
    xp = cur == 0 ? a.xb[2] : (cur == 1 ? a.xb[0] : a.xb[1]);
    beta = (float)(a.gm + gi_)->beta;
  } else {
    x = a.x;
    xp = a.xprev;
    beta = a.beta;
  }
  const int s = bid_ / NB, rb = bid_ % NB;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31, rl = warp >> 1, j = warp & 1;
  const size_t base = g.img_off + ((size_t)s * N + rb * RB + rl) * N;
  // packed row z[m] = y[2m] + i y[2m+1], m < 1024 (the padding above is zero), times w^(jm)
  float2 v[P];
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const int m = t + T * i;
    const float2 xv = __ldg(reinterpret_cast<const float2*>(x + base) + m);
    const float2 pv = __ldg(reinterpret_cast<const float2*>(xp + base) + m);
    float2 z = make_float2(fmaf(beta, xv.x - pv.x, xv.x), fmaf(beta, xv.y - pv.y, xv.y));
    if (j) z = cmul(z, __ldg(&g.twM[2 * m]));  // w^m = W^(2m)
    v[i] = z;
  });
  Q::F::template run<-1, float2, 2>(v, sm + warp * Q::F::SMEM, g.twN, t);
  __syncthreads();  // every exchange buffer is free: the staged rows alias them
  float2* zrow = sm + rl * LDZ;
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    zrow[2 * (t + T * i) + j] = v[i];
  });
  __syncthreads();
  // split Y[v] = E[v] + W^v O[v] with E = (Z[v] + conj Z[N - v]) / 2, O = (Z[v] - conj Z[N - v]) / 2i,
  // two mirrored outputs at a time: E[N - v] = conj E[v], O[N - v] = conj O[v] and
  // W^(N - v) = -conj W^v give Y[N - v] = conj(E[v] - W^v O[v]) (v = 0: Y[N] = Re Z[0] - Im Z[0]);
  // written column-major (RB-row segments)
  using IO = SpecIO<BF>;
  typename IO::T* out = reinterpret_cast<typename IO::T*>(g.spec) + (size_t)s * (N + 1) * N + rb * RB;
  for (int e = threadIdx.x; e < (N / 2 + 1) * RB; e += THREADS) {
    const int vv = e / RB, rr = e - vv * RB;
    const float2* zr = sm + rr * LDZ;
    const float2 z = zr[vv], zs = zr[(N - vv) & (N - 1)];
    const float2 ev = make_float2(0.5f * (z.x + zs.x), 0.5f * (z.y - zs.y));
    const float2 od = make_float2(0.5f * (z.y + zs.y), -0.5f * (z.x - zs.x));
    const float2 wo = cmul(__ldg(&g.twM[vv]), od);
    IO::st(out, (size_t)vv * N + rr, cadd(ev, wo));
    if (vv != N / 2) IO::st(out, (size_t)(N - vv) * N + rr, make_float2(ev.x - wo.x, wo.y - ev.y));
  }
}

template <bool BF>
__global__ void __launch_bounds__(128, 3) k_pass2_q(const __grid_constant__ GroupSet gs, const IterState* st) {
  using Q = Q2048;
  constexpr int N = Q::N, H = Q::H, T = 32, P = 32;
  extern __shared__ float2 sm[];
  int bid_;
  const int gi_ = gs.pick(bid_);
  const GroupDev& g = gs.g[gi_];
  if (st && skip_iter<BF>(st)) return;
  const int j = threadIdx.x >> 5, t = threadIdx.x & 31;
  int vcol, s;
  column_of(bid_, g.S, N + 1, vcol, s);
  using IO = SpecIO<BF>;
  typename IO::T* p = reinterpret_cast<typename IO::T*>(g.spec) + ((size_t)s * (N + 1) + vcol) * N;
  float2* col = sm;
  if constexpr (!BF) {
    // all of the column's copies in flight at once
    SFor<0, N / 128>::run([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      tc05::cp_async8(&col[threadIdx.x + 128 * i], p + threadIdx.x + 128 * i);
    });
    tc05::cp_async_wait_all();
  } else {
    batched_copy<128, 16>(N, [&](int r) { return IO::ld(p, r); }, [&](int r, float2 v) { col[r] = v; });
  }
  __syncthreads();
  float2 v[P];
  // y_j[m] = W^(jm) (c[m] + (-i)^j c[m + 1024]) with m = t + 32 i; W^(jm) = W^(jt) W^(32 j i), the
  // first factor one table read per thread, the second a compile-time constant per element
  auto prologue = [&](auto J_) {
    constexpr int J = decltype(J_)::value;
    const float2 base = tw4096(g.twM, J * t);
    SFor<0, P>::run([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      const int m = t + T * i;
      const float2 a0 = col[m], b = col[m + H];
      float2 c;
      if constexpr (J == 0)
        c = cadd(a0, b);
      else if constexpr (J == 1)
        c = make_float2(a0.x + b.y, a0.y - b.x);  // a + (-i) b
      else if constexpr (J == 2)
        c = csub(a0, b);
      else
        c = make_float2(a0.x - b.y, a0.y + b.x);  // a + i b
      if constexpr (J != 0) c = cmul(c, twmul<32 * J * i, 4096, -1>(base));
      v[i] = c;
    });
  };
  switch (j) {
    case 0: prologue(std::integral_constant<int, 0>{}); break;
    case 1: prologue(std::integral_constant<int, 1>{}); break;
    case 2: prologue(std::integral_constant<int, 2>{}); break;
    default: prologue(std::integral_constant<int, 3>{}); break;
  }
  float2* xs = sm + N + j * Q::F::SMEM;
  Q::F::template run<-1, float2, 2>(v, xs, g.twN, t);
  // v[i] = X[4k + j], k = t + 32 i: row 4k + j of the 2N grid is row 2k + (j >> 1) of the
  // (j & 1) half of the kernel spectrum
  const float* cc = g.chat + ((size_t)vcol * 2 + (j & 1)) * N + (j >> 1);
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const float c = __ldg(&cc[2 * (t + T * i)]);
    v[i] = make_float2(v[i].x * c, v[i].y * c);
  });
  Q::F::template run<1, float2, 2>(v, xs, g.twN, t);
  __syncwarp();  // the transform's last exchange reads are done: the buffer takes W^(-jm) u_j
  auto epilogue = [&](auto J_) {
    constexpr int J = decltype(J_)::value;
    const float2 base = tw4096(g.twM, J * t);
    SFor<0, P>::run([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      if constexpr (J == 0)
        xs[t + T * i] = v[i];
      else
        xs[t + T * i] = cmulc(v[i], twmul<32 * J * i, 4096, -1>(base));
    });
  };
  switch (j) {
    case 0: epilogue(std::integral_constant<int, 0>{}); break;
    case 1: epilogue(std::integral_constant<int, 1>{}); break;
    case 2: epilogue(std::integral_constant<int, 2>{}); break;
    default: epilogue(std::integral_constant<int, 3>{}); break;
  }
  __syncthreads();
  // kept rows: z[m] = v_0 + v_1 + v_2 + v_3, z[m + 1024] = (v_0 - v_2) + i (v_1 - v_3)
  const float2* b0 = sm + N;
  for (int m = threadIdx.x; m < H; m += 128) {
    const float2 a0 = b0[m], a1 = b0[Q::F::SMEM + m], a2 = b0[2 * Q::F::SMEM + m], a3 = b0[3 * Q::F::SMEM + m];
    const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
    IO::st(p, m, cadd(s02, s13));
    IO::st(p, m + H, make_float2(d02.x - d13.y, d02.y + d13.x));
  }
}

template <bool BF, int RB>
__global__ void __launch_bounds__(64 * RB, 8 / RB) k_pass3a_q(const __grid_constant__ GroupSet gs, const IterState* st, float* apply_out) {
  using Q = Q2048;
  constexpr int N = Q::N, T = 32, P = 32, LDZ = Q::LDZ, THREADS = 64 * RB, NB = N / RB;
  extern __shared__ float2 sm[];
  int bid_;
  const int gi_ = gs.pick(bid_);
  const GroupDev& g = gs.g[gi_];
  float* kz = apply_out ? apply_out + g.img_off : g.kz;
  if (st && skip_iter<BF>(st)) return;
  const int s = bid_ / NB, rb = bid_ % NB;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31, rl = warp >> 1, j = warp & 1;
  const int r0 = rb * RB;
  {
    using IO = SpecIO<BF>;
    const typename IO::T* sp = reinterpret_cast<const typename IO::T*>(g.spec) + (size_t)s * (N + 1) * N + r0;
    if constexpr (!BF) {
      // RB-row segments of the column-major spectrum, all copies in flight at once
      for (int e = threadIdx.x; e < (N + 1) * RB; e += THREADS) {
        const int vv = e / RB, rr = e - vv * RB;
        tc05::cp_async8(&sm[rr * LDZ + vv], sp + (size_t)vv * N + rr);
      }
      tc05::cp_async_wait_all();
    } else {
      batched_copy<THREADS, 8>(
          (N + 1) * RB, [&](int e) { return IO::ld(sp, (size_t)(e / RB) * N + e % RB); },
          [&](int e, float2 v) { sm[(e % RB) * LDZ + e / RB] = v; });
    }
  }
  __syncthreads();
  // the length-2N real inverse as the length-N complex inverse of Z[v] = E[v] + i O[v], at the
  // v = 2k + j of this warp
  float2 q[P];
  const float2* row = sm + rl * LDZ;
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const int vp = 2 * (t + T * i) + j;
    const float2 zv = row[vp], zr = row[N - vp];
    const float2 e = make_float2(zv.x + zr.x, zv.y - zr.y);
    const float2 d = make_float2(zv.x - zr.x, zv.y + zr.y);
    const float2 o = cmulc(d, __ldg(&g.twM[vp]));
    q[i] = make_float2(e.x - o.y, e.y + o.x);
  });
  __syncthreads();  // the staged rows are read: the exchange buffers alias them
  float2* xs = sm + warp * Q::F::SMEM;
  Q::F::template run<1, float2, 2>(q, xs, g.twN, t);
  __syncwarp();
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const int n = t + T * i;
    xs[n] = j ? cmulc(q[i], __ldg(&g.twM[2 * n])) : q[i];  // w^(-jn) u_j[n]
  });
  __syncthreads();
  // z[n] = sum_j w^(-jn) u_j[n]: each warp of the row sums one half of it
  const float2* o0 = sm + (2 * rl) * Q::F::SMEM;
  float2* out = reinterpret_cast<float2*>(kz + ((size_t)s * N + r0 + rl) * N);
  for (int n = j * (Q::H / 2) + t; n < (j + 1) * (Q::H / 2); n += 32) out[n] = cadd(o0[n], o0[Q::F::SMEM + n]);
}

// ---------------------------------------------------------------- pass 3b: gradient and update
// The prior gradient of Eq. 5 at voxel v is sum_o w_o rho'(y_v - y_{v+o}) over the 26
// neighbours; rho' is odd, so the pair (v, v+o) adds +f to v and -f to v+o.  Every unordered
// pair is evaluated once, from its lexicographically smaller end (13 forward offsets), and
// the value is handed to the other end instead of being recomputed there.
//
// A block owns R = 4 rows (a band) by BC columns of one group and marches through a chunk of
// its slices.  Warp w owns 64 columns; lane l owns the voxel pair a = 2l, b = 2l + 1 of every
// row of the band as the two lanes of packed FP32 pairs, so the pair (a, b) stays in the
// thread, the pairs with columns a - 1 and b + 1 go to the neighbouring lanes by shuffle, and
// the pairs that cross a warp's outer columns are evaluated once more by the receiving warp
// (nine per row, spread over the lanes before the row walk).  Rows are walked top to bottom
// with the halo rows -1 and R as sources of pairs into the band; slice z is the source of
// the pairs into slice z + 1, whose contributions wait in shared memory (one entry per
// thread) for the next step.  A chunk starting at z0 > 0 first evaluates the pairs between
// slices z0 - 1 and z0 (the only pairs evaluated twice, once per chunk).  Shared memory holds
// y for slices z and z + 1 (rows -1 .. R, columns c0 - 4 .. c0 + BC + 3), each beside a copy
// shifted by one column so that the neighbour pairs (a - 1, a) and (b, b + 1) are aligned 8-byte
// loads like (a, b); x and x_prev of slice z + 2, arriving by asynchronous copies while slice
// z is worked on; the carried contributions; and K (*) y, R*g and x_k at each thread's voxels,
// copied asynchronously one slice ahead.  Neighbours outside the volume read the voxel itself
// (d = 0 adds nothing).
template <int N>
struct GeoP {
  static_assert(N % 64 == 0, "a warp owns 64 columns");
  static constexpr int R = 4;                             // rows of a band
  static constexpr int WPB = N / 64 < 8 ? N / 64 : 8;     // warps per block
  static constexpr int THREADS = 32 * WPB;
  static constexpr int BC = 64 * WPB;                     // columns of a block
  static constexpr int CB = N / BC;                       // column blocks per band
  static constexpr int NB = N / R;                        // bands per slice
  static constexpr int LDR = BC + 8;                      // ring row stride (floats)
  static constexpr int RING = (R + 2) * LDR;              // y of one slice (the shifted copy follows)
  static constexpr int NEDGE = 9 * R;                     // cross-warp pairs per warp and step
  static constexpr int FIN = 3 * R * THREADS;            // K (*) y, R*g, x_k of the band (float2)
  // ring (2 slices of y and shifted y) | staging (x, x_prev of one slice) | carry | cross-warp
  // pair values | the next slice's K (*) y, R*g and x_k at each thread's voxels
  static constexpr size_t SM = (size_t)(6 * RING + R * BC + WPB * NEDGE) * sizeof(float) + (size_t)FIN * 8;
  static_assert(N % BC == 0, "column blocks");
};

// y = x + beta (x - x_prev) of one slice, rows r0 - 1 .. r0 + R, columns c0 - 4 .. c0 + BC + 3,
// into a ring slot (zero outside the image)
template <int N>
__device__ __forceinline__ void load_ring_p(float* slot, const float* x, const float* xp, float beta,
                                            size_t off_slice, int r0, int c0) {
  using GP = GeoP<N>;
  constexpr int Q = GP::LDR / 4;
  for (int e = threadIdx.x; e < (GP::R + 2) * Q; e += GP::THREADS) {
    const int q = e % Q, rowi = e / Q;
    const int rr = r0 - 1 + rowi, cc = c0 - 4 + 4 * q;
    float4 yv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (rr >= 0 && rr < N && cc >= 0 && cc < N) {
      const size_t off = off_slice + (size_t)rr * N + cc;
      const float4 xv = __ldg(reinterpret_cast<const float4*>(x + off));
      const float4 pv = __ldg(reinterpret_cast<const float4*>(xp + off));
      yv = make_float4(fmaf(beta, xv.x - pv.x, xv.x), fmaf(beta, xv.y - pv.y, xv.y), fmaf(beta, xv.z - pv.z, xv.z),
                       fmaf(beta, xv.w - pv.w, xv.w));
    }
    reinterpret_cast<float4*>(slot + rowi * GP::LDR)[q] = yv;
  }
}

// x and x_prev of one slice (the ring's rows and columns) into the staging area by
// asynchronous 16-byte copies, zero-filled outside the image
template <int N>
__device__ __forceinline__ void stage_issue(float* stg, const float* x, const float* xp, size_t off_slice, int r0,
                                            int c0) {
  using GP = GeoP<N>;
  constexpr int Q = GP::LDR / 4;
  for (int e = threadIdx.x; e < (GP::R + 2) * Q; e += GP::THREADS) {
    const int q = e % Q, rowi = e / Q;
    const int rr = r0 - 1 + rowi, cc = c0 - 4 + 4 * q;
    const bool ok = rr >= 0 && rr < N && cc >= 0 && cc < N;
    const size_t off = ok ? off_slice + (size_t)rr * N + cc : off_slice;
    tc05::cp_async16(stg + 4 * e, x + off, ok);
    tc05::cp_async16(stg + GP::RING + 4 * e, xp + off, ok);
  }
}
// y = x + beta (x - x_prev) from the staging area into a ring slot, and the copy shifted by
// one column (shifted[i] = y[i + 1]) after it
template <int N>
__device__ __forceinline__ void stage_to_ring(float* slot, const float* stg, float beta) {
  using GP = GeoP<N>;
  for (int e = threadIdx.x; e < GP::RING / 4; e += GP::THREADS) {
    const float4 xv = reinterpret_cast<const float4*>(stg)[e];
    const float4 pv = reinterpret_cast<const float4*>(stg + GP::RING)[e];
    const float4 y =
        make_float4(fmaf(beta, xv.x - pv.x, xv.x), fmaf(beta, xv.y - pv.y, xv.y), fmaf(beta, xv.z - pv.z, xv.z),
                    fmaf(beta, xv.w - pv.w, xv.w));
    float nx = 0.f;
    if (4 * e + 4 < GP::RING) {
      const float x4 = stg[4 * e + 4], p4 = stg[GP::RING + 4 * e + 4];
      nx = fmaf(beta, x4 - p4, x4);
    }
    reinterpret_cast<float4*>(slot)[e] = y;
    reinterpret_cast<float4*>(slot + GP::RING)[e] = make_float4(y.y, y.z, y.w, nx);
  }
}
// the shifted copy of a ring slot whose y part is in place
template <int N>
__device__ __forceinline__ void ring_shift(float* slot) {
  using GP = GeoP<N>;
  for (int e = threadIdx.x; e < GP::RING / 4; e += GP::THREADS) {
    const float4 v = reinterpret_cast<const float4*>(slot)[e];
    const float nx = 4 * e + 4 < GP::RING ? slot[4 * e + 4] : 0.f;
    reinterpret_cast<float4*>(slot + GP::RING)[e] = make_float4(v.y, v.z, v.w, nx);
  }
}

// The lane's neighbour pair at column offset DX in a ring row (y part; the shifted copy sits
// RING floats further): DX = -1: (y[a - 1], y[a]), 0: (y[a], y[b]), +1: (y[b], y[b + 1]).
// A neighbour outside the image reads the voxel itself: with ROWE for a missing row (row_ok
// false), with COLE for a missing column a - 1 or b + 1.
template <int N, int DX, bool ROWE, bool COLE>
__device__ __forceinline__ float2 nb_pair(const float* row, int ia, float2 y, bool row_ok, bool okL, bool okR) {
  constexpr int RING = GeoP<N>::RING;
  float2 n;
  if constexpr (DX < 0)
    n = *reinterpret_cast<const float2*>(row + RING + ia - 2);
  else if constexpr (DX == 0)
    n = *reinterpret_cast<const float2*>(row + ia);
  else
    n = *reinterpret_cast<const float2*>(row + RING + ia);
  if constexpr (COLE) {
    if constexpr (DX < 0) n.x = okL ? n.x : y.x;
    if constexpr (DX > 0) n.y = okR ? n.y : y.y;
  }
  if constexpr (ROWE) n = row_ok ? n : y;
  return n;
}

// Weighted pair value f = w sigma^2 rho'(y - nb) / sigma^2 of two pairs at once (the weight
// arrives as wq = w (q - p) / sigma^2, wp = w p / sigma^2), with the identity of nbr2:
// sigma^2 rho'(d) = d |d/sigma|^(q-2) r (p + (q - p) r), r = 1 / (1 + |d/(c sigma)|^(q-p)).
// With PH, ph += sigma^2 rho(d) = d^2 |d/sigma|^(q-2) r (unweighted).
template <bool Q2, bool PH>
__device__ __forceinline__ float2 pairv(float2 y, float2 nb, const PriorK& k, float2 wq, float2 wp, float2& ph) {
  const float2 d = f2fma(nb, f2(-1.f), y);
  const float2 sq = f2fma(d, d, f2(1e-30f));
  const float2 la = make_float2(lg2a(sq.x), lg2a(sq.y));
  const float2 s = f2fma(k.half_qp, la, k.qp_l2);
  const float2 e = f2add(make_float2(ex2a(s.x), ex2a(s.y)), f2(1.f));
  const float2 r = make_float2(rcpa(e.x), rcpa(e.y));
  float2 dr = f2mul(d, r);
  if constexpr (!Q2) {
    const float2 s2 = f2fma(k.half_q2, la, k.q2_l2);
    dr = f2mul(dr, make_float2(ex2a(s2.x), ex2a(s2.y)));
  }
  if constexpr (PH) ph = f2fma(d, dr, ph);
  return f2mul(dr, f2fma(wq, r, wp));
}

// hi + lo += v with the rounding error of the addition kept in lo (Knuth's TwoSum): the
// per-slice partial sums stay in FP32, whose pipe is wide, instead of FP64, whose is not
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}

// Block reduction of compensated FP32 sums (hi + lo per thread) to partials[block]: TwoSum
// across each warp, FP64 across the warps, in a fixed order.
template <int W>
__device__ __forceinline__ void block_partials_f(float (&hi)[kParts], float (&lo)[kParts], double* red,
                                                 double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kParts; ++j) {
    float h = hi[j], l = lo[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_down_sync(0xffffffffu, h, o), l2 = __shfl_down_sync(0xffffffffu, l, o);
      l += l2;
      two_sum_add(h, l, h2);
    }
    if (lane == 0) red[warp * kParts + j] = (double)h + (double)l;
  }
  __syncthreads();
  if (threadIdx.x < kParts) {
    double sum = 0.0;
    for (int w = 0; w < W; ++w) sum += red[w * kParts + threadIdx.x];
    out[threadIdx.x] = sum;
  }
}

// class weights of the pair values: wq = w (q - p) / sigma^2, wp = w p / sigma^2 for the face,
// edge and corner neighbours
struct PairW {
  float2 wq[3], wp[3];
};

// the three pairs (+1, DY, -1 / 0 / +1) from source voxels (a, b) into ring row T of the next
// slice: +f to the source, -f to the target (own lanes) or sent to the lane that owns it
template <int N, bool Q2, bool PH, bool ROWE, bool COLE, int DY>
__device__ __forceinline__ void cross3(float2 y, const float* T, int ia, bool rok, bool okL, bool okR,
                                       const PriorK& k, const PairW& pw, float2& gsrc, float2& C, float& sR,
                                       float& sL, float2 (&phr)[3]) {
  constexpr int CS = DY == 0 ? 1 : 2;  // class of the dx = -1, +1 pairs
  constexpr int C0 = DY == 0 ? 0 : 1;  // class of the dx = 0 pair
  float2 f = pairv<Q2, PH>(y, nb_pair<N, -1, ROWE, COLE>(T, ia, y, rok, okL, okR), k, pw.wq[CS], pw.wp[CS], phr[CS]);
  gsrc = f2add(gsrc, f);
  sL += f.x;
  C.x -= f.y;
  f = pairv<Q2, PH>(y, nb_pair<N, 0, ROWE, COLE>(T, ia, y, rok, okL, okR), k, pw.wq[C0], pw.wp[C0], phr[C0]);
  gsrc = f2add(gsrc, f);
  C = f2fma(f, f2(-1.f), C);
  f = pairv<Q2, PH>(y, nb_pair<N, 1, ROWE, COLE>(T, ia, y, rok, okL, okR), k, pw.wq[CS], pw.wp[CS], phr[CS]);
  gsrc = f2add(gsrc, f);
  C.y -= f.x;
  sR += f.y;
}

// One slice step of a band: every pair whose source voxel lies in slice zs (ring slot S0) and
// whose other end lies in zs or zs + 1 (slot S1, when have1).  The carried contributions of
// slice zs (cr, this thread's entries, row stride BC / 2) start the gradient rows and are
// replaced by those of slice zs + 1.  PRE: only the pairs into slice zs + 1 (a chunk start);
// otherwise each owned row t is handed to fin(t, gradient sum, y) once complete, with ph the
// unweighted sigma^2 rho sums by class of the pairs the band owns.  ROWE: the band is the
// image's first or last; COLE: the warp holds its first or last 64 columns.  Elsewhere every
// neighbour lies inside the image and the boundary tests drop out.
template <int N, bool Q2, bool PHI, bool PRE, bool ROWE, bool COLE, class Fin>
__device__ __forceinline__ void band_step(const float* S0, const float* S1, bool have1, int r0, int c0w, int ia,
                                          bool okL_, bool okR_, float2* cr, float* edge, const PriorK& k,
                                          const PairW& pw, float2 (&ph)[3], Fin&& fin) {
  using GP = GeoP<N>;
  constexpr int R = GP::R, LDR = GP::LDR, HALF = GP::NEDGE / 2, CRS = GP::BC / 2;
  constexpr bool PH = PHI && !PRE;
  const int lane = threadIdx.x & 31;
  const int cw = ia - 4 - 2 * lane;  // ring column of the warp's first column, minus 4
  const bool top = !ROWE || r0 > 0, bot = !ROWE || r0 + R < N;
  const bool okL = !COLE || okL_, okR = !COLE || okR_;

  // ---- pairs across the warp's outer columns, evaluated by the receiving warp.  Item
  // kd * R + t is one pair into column c0w (kd < 5) or c0w + 63 (kd >= 5) of row t:
  //   kd 0: (0, 0, +1) from row t       kd 5: (0, +1, -1) from row t - 1
  //   kd 1: (0, +1, +1) from row t - 1  kd 6..8: (+1, -1 / 0 / +1, -1) from rows t + 1, t, t - 1
  //   kd 2..4: (+1, -1 / 0 / +1, +1) from rows t + 1, t, t - 1
  // (kd 2..4 and 6..8 land in slice zs + 1).  Two items per lane; slot = -f for the target.
  if (lane < HALF) {
    float ys[2], yt[2], wq[2], wp[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + h * HALF;
      const int kd = i / R, t = i - kd * R;
      const bool left = kd < 5;
      const int sr = (kd == 0 || kd == 3 || kd == 7) ? 0 : ((kd == 2 || kd == 6) ? 1 : -1);
      const bool cross = kd >= 2 && kd != 5;
      const int cls = kd == 0 ? 0 : ((kd & 1) ? 1 : 2);
      const int tr = t + sr;
      const bool ok = (!ROWE || (r0 + tr >= 0 && r0 + tr < N)) && (!COLE || (left ? c0w > 0 : c0w + 64 < N)) &&
                      (cross ? have1 : !PRE);
      const float tv = (cross ? S1 : S0)[(t + 1) * LDR + cw + (left ? 4 : 67)];
      const float sv = S0[(tr + 1) * LDR + cw + (left ? 3 : 68)];
      ys[h] = ok ? sv : tv;
      yt[h] = tv;
      wq[h] = cls == 0 ? pw.wq[0].x : (cls == 1 ? pw.wq[1].x : pw.wq[2].x);
      wp[h] = cls == 0 ? pw.wp[0].x : (cls == 1 ? pw.wp[1].x : pw.wp[2].x);
    }
    float2 unused;
    const float2 f = pairv<Q2, false>(make_float2(ys[0], ys[1]), make_float2(yt[0], yt[1]), k,
                                      make_float2(wq[0], wq[1]), make_float2(wp[0], wp[1]), unused);
    edge[lane] = -f.x;
    edge[lane + HALF] = -f.y;
  }
  __syncwarp();

  // ---- the row walk: source rows -1 .. R of slice zs (ring row t + 1 holds image row r0 + t),
  // unrolled at compile time so that the row tests and the window slides cost nothing
  const float2 zero = f2(0.f);
  float2 gc = zero, gn = PRE ? zero : cr[0];                                // gradient rows t, t + 1
  float2 cm = zero, cc = zero, cp = zero;                                   // carry rows t - 1, t, t + 1
  float sRc = 0.f, sRn = 0.f, sLc = 0.f, sLn = 0.f;                         // sends into rows t, t + 1
  float sR1m = 0.f, sR1c = 0.f, sR1p = 0.f, sL1m = 0.f, sL1c = 0.f, sL1p = 0.f;
  SFor<-1, R + 1>::run([&](auto t_) {
    constexpr int t = decltype(t_)::value;
    constexpr bool own = t >= 0 && t < R;
    const float* rowt = S0 + (t + 1) * LDR;  // slice zs, row t
    const float2 y = *reinterpret_cast<const float2*>(rowt + ia);
    float2 phr[3] = {zero, zero, zero};
    if constexpr (!PRE && own) {  // (0, 0, +1), face
      const float2 f = pairv<Q2, PH>(y, nb_pair<N, 1, ROWE, COLE>(rowt, ia, y, true, okL, okR), k, pw.wq[0], pw.wp[0],
                                     phr[0]);
      gc = f2add(gc, f);
      gc.y -= f.x;
      sRc += f.y;
    }
    if constexpr (!PRE && t < R) {
      if (own || top) {  // (0, +1, -1 / 0 / +1) into row t + 1
        const bool rok = !ROWE || r0 + t + 1 < N;
        const float* rown = rowt + LDR;
        float2 f = pairv<Q2, PH>(y, nb_pair<N, -1, ROWE, COLE>(rown, ia, y, rok, okL, okR), k, pw.wq[1], pw.wp[1], phr[1]);
        gc = f2add(gc, f);
        sLn += f.x;
        gn.x -= f.y;
        f = pairv<Q2, PH>(y, nb_pair<N, 0, ROWE, COLE>(rown, ia, y, rok, okL, okR), k, pw.wq[0], pw.wp[0], phr[0]);
        gc = f2add(gc, f);
        gn = f2fma(f, f2(-1.f), gn);
        f = pairv<Q2, PH>(y, nb_pair<N, 1, ROWE, COLE>(rown, ia, y, rok, okL, okR), k, pw.wq[1], pw.wp[1], phr[1]);
        gc = f2add(gc, f);
        gn.y -= f.x;
        sRn += f.y;
      }
    }
    if (have1) {  // (+1, dy, dx) into rows t - 1, t, t + 1 of slice zs + 1
      if constexpr (t >= 0) {
        if (own || bot)
          cross3<N, Q2, PH, ROWE, COLE, -1>(y, S1 + t * LDR, ia, !ROWE || r0 + t - 1 >= 0, okL, okR, k, pw, gc, cm, sR1m,
                                      sL1m, phr);
      }
      if constexpr (own)
        cross3<N, Q2, PH, ROWE, COLE, 0>(y, S1 + (t + 1) * LDR, ia, true, okL, okR, k, pw, gc, cc, sR1c, sL1c, phr);
      if constexpr (t < R) {
        if (own || top)
          cross3<N, Q2, PH, ROWE, COLE, 1>(y, S1 + (t + 2) * LDR, ia, !ROWE || r0 + t + 1 < N, okL, okR, k, pw, gc, cp,
                                     sR1p, sL1p, phr);
      }
    }
    if constexpr (PH && own) {
#pragma unroll
      for (int j = 0; j < 3; ++j) ph[j] = f2add(ph[j], phr[j]);
    }
    // gradient row t (in-plane sources t - 1, t) and carry row t - 1 (sources t - 2 .. t) are
    // complete: take the neighbouring lanes' shares
    if constexpr (!PRE && own) {
      const float rx = __shfl_up_sync(0xffffffffu, sRc, 1), lx = __shfl_down_sync(0xffffffffu, sLc, 1);
      gc.x -= lane > 0 ? rx : 0.f;
      gc.y -= lane < 31 ? lx : 0.f;
      if (lane == 0) gc.x += edge[t] + edge[R + t];
      if (lane == 31) gc.y += edge[5 * R + t];
      fin(t, gc, y);
    }
    if constexpr (t >= 1) {
      const float rx1 = __shfl_up_sync(0xffffffffu, sR1m, 1), lx1 = __shfl_down_sync(0xffffffffu, sL1m, 1);
      cm.x -= lane > 0 ? rx1 : 0.f;
      cm.y -= lane < 31 ? lx1 : 0.f;
      if (lane == 0) cm.x += edge[2 * R + t - 1] + edge[3 * R + t - 1] + edge[4 * R + t - 1];
      if (lane == 31) cm.y += edge[6 * R + t - 1] + edge[7 * R + t - 1] + edge[8 * R + t - 1];
      cr[(t - 1) * CRS] = cm;
    }
    // slide the windows down one row
    gc = gn;
    if constexpr (!PRE && t + 2 < R)
      gn = cr[(t + 2) * CRS];
    else
      gn = zero;
    sRc = sRn;
    sRn = 0.f;
    sLc = sLn;
    sLn = 0.f;
    cm = cc;
    cc = cp;
    cp = zero;
    sR1m = sR1c;
    sR1c = sR1p;
    sR1p = 0.f;
    sL1m = sL1c;
    sL1c = sL1p;
    sL1p = 0.f;
  });
}

// kz: K (*) y of the group from pass 3a ([slice][row][col]); phase: in Iterate mode, the storage
// phase this launch belongs to (0 FP32, 1 BF16), checked like the other passes.
template <int N, int MODE, bool Q2, bool MULTI>
__global__ void __launch_bounds__(GeoP<N>::THREADS, 2)
    k_pass3(const __grid_constant__ GroupSet gs, StepArgs a, PriorC pc, const float* apply_out, int phase,
            double* partials, int block_offset) {
  using GP = GeoP<N>;
  constexpr int R = GP::R;
  constexpr bool PRIOR = MODE != (int)Pass3Mode::Apply;
  constexpr bool PHI = MODE == (int)Pass3Mode::Step || MODE == (int)Pass3Mode::Iterate ||
                       MODE == (int)Pass3Mode::Objective;
  constexpr bool UPDATE = MODE == (int)Pass3Mode::Step || MODE == (int)Pass3Mode::Iterate;
  extern __shared__ float2 sm[];
  __shared__ double red[GP::WPB * kParts];
  int bid_;
  const int gi_ = gs.template pick<MULTI>(bid_);
  const GroupDev& g = gs.g[MULTI ? gi_ : 0];
  const float* __restrict__ kz = apply_out ? apply_out + g.img_off : g.kz;
  const int zc = g.zc;  // resolved by the launcher
  const float *x, *xp;
  float* out;
  float beta, invL;
  if constexpr (MODE == (int)Pass3Mode::Iterate) {
    if (a.st->done || a.st->bf16 != phase) return;
    const int cur = a.st->cur;
    x = cur == 0 ? a.xb[0] : (cur == 1 ? a.xb[1] : a.xb[2]);
    xp = cur == 0 ? a.xb[2] : (cur == 1 ? a.xb[0] : a.xb[1]);
    out = cur == 0 ? a.xb[1] : (cur == 1 ? a.xb[2] : a.xb[0]);
    beta = (float)(a.gm + gi_)->beta;
    invL = (float)(a.gm + gi_)->invL;
  } else {
    x = a.x;
    xp = a.xprev;
    out = a.out;
    beta = a.beta;
    invL = a.invL;
  }
  // the group's slices as the origin of every image pointer
  const size_t go = g.img_off;
  const int S = g.S;
  x += go;
  xp += go;
  out += go;
  const float* __restrict__ atg = a.atg + go;
  const int band = bid_ % GP::NB;
  const int cb = (bid_ / GP::NB) % GP::CB;
  const int chunk = bid_ / (GP::NB * GP::CB);
  const int z0 = g.zlo + chunk * zc, z1 = min(g.zlo + (g.zn > 0 ? g.zn : S), z0 + zc);
  const int r0 = band * R, c0 = cb * GP::BC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0w = c0 + 64 * warp;
  const int acol = c0w + 2 * lane;  // this lane's voxels: columns acol, acol + 1
  const int ia = 64 * warp + 2 * lane + 4;
  const size_t N2 = (size_t)N * N;

  float hi[kParts], lo[kParts];  // compensated FP32 sums of the block's slices
#pragma unroll
  for (int j = 0; j < kParts; ++j) hi[j] = lo[j] = 0.f;

  if constexpr (!PRIOR) {
    // Apply: pass 3a wrote K (*) x to the output itself; only the partial sums remain
    for (int z = z0; z < z1; ++z) {
      float2 acc0 = f2(0.f), acc5 = f2(0.f);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const size_t o = (size_t)z * N2 + (size_t)(r0 + t) * N + acol;
        const float2 zd = __ldg(reinterpret_cast<const float2*>(kz + o));
        const float2 xv = __ldg(reinterpret_cast<const float2*>(x + o));
        acc0 = f2fma(xv, zd, acc0);
        acc5 = f2fma(zd, zd, acc5);
      }
      two_sum_add(hi[0], lo[0], acc0.x + acc0.y);
      two_sum_add(hi[5], lo[5], acc5.x + acc5.y);
    }
  } else {
    const PriorK pk = prior_k(pc);
    PairW pw;
    const float wcls[3] = {pc.wf * pc.inv_sig2, pc.we * pc.inv_sig2, pc.wc * pc.inv_sig2};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      pw.wq[j] = f2(wcls[j] * pc.qp);
      pw.wp[j] = f2(wcls[j] * pc.p);
    }
    const float2 lam = f2(pc.lam);
    const bool okL = acol > 0, okR = acol + 2 < N;
    float* ring = reinterpret_cast<float*>(sm);
    constexpr int SLOT = 2 * GP::RING;  // y and its shifted copy
    float* stg = ring + 2 * SLOT;
    float2* cr = reinterpret_cast<float2*>(stg + 2 * GP::RING) + 32 * warp + lane;
    float* edge = stg + 2 * GP::RING + R * GP::BC + warp * GP::NEDGE;
    float2* fin_in = reinterpret_cast<float2*>(stg + 2 * GP::RING + R * GP::BC + GP::WPB * GP::NEDGE) + threadIdx.x;
    // K (*) y, R*g and x_k of row t of slice zz at this thread's voxels, into fin_in
    auto fetch = [&](int zz, int t) {
      const size_t o = (size_t)zz * N2 + (size_t)(r0 + t) * N + acol;
      float2* d = fin_in + 3 * t * GP::THREADS;
      tc05::cp_async8(d, kz + o);
      tc05::cp_async8(d + GP::THREADS, atg + o);
      if constexpr (UPDATE) tc05::cp_async8(d + 2 * GP::THREADS, x + o);
    };
    float2 ph[3] = {f2(0.f), f2(0.f), f2(0.f)};
    load_ring_p<N>(ring + (z0 & 1) * SLOT, x, xp, beta, (size_t)z0 * N2, r0, c0);
    if (z0 > 0) {
      load_ring_p<N>(ring + ((z0 - 1) & 1) * SLOT, x, xp, beta, (size_t)(z0 - 1) * N2, r0, c0);
    } else {
#pragma unroll
      for (int t = 0; t < R; ++t) cr[t * (GP::BC / 2)] = f2(0.f);
    }
    __syncthreads();
    ring_shift<N>(ring + (z0 & 1) * SLOT);
    if (z0 > 0) ring_shift<N>(ring + ((z0 - 1) & 1) * SLOT);
    if (z0 + 1 < S) stage_issue<N>(stg, x, xp, (size_t)(z0 + 1) * N2, r0, c0);
#pragma unroll
    for (int t = 0; t < R; ++t) fetch(z0, t);
    __syncthreads();
    // boundary tests only where the warp's neighbourhoods leave the image
    const bool rowe = !(r0 > 0 && r0 + R < N), cole = !(c0w > 0 && c0w + 64 < N);
    if (z0 > 0) {
      auto fin0 = [](int, float2, float2) {};
      const float* s0 = ring + ((z0 - 1) & 1) * SLOT;
      const float* s1 = ring + (z0 & 1) * SLOT;
      if (rowe)
        band_step<N, Q2, PHI, true, true, true>(s0, s1, true, r0, c0w, ia, okL, okR, cr, edge, pk, pw, ph, fin0);
      else if (cole)
        band_step<N, Q2, PHI, true, false, true>(s0, s1, true, r0, c0w, ia, okL, okR, cr, edge, pk, pw, ph, fin0);
      else
        band_step<N, Q2, PHI, true, false, false>(s0, s1, true, r0, c0w, ia, okL, okR, cr, edge, pk, pw, ph, fin0);
    }
    for (int z = z0; z < z1; ++z) {
      // every thread has finished slice z - 1, so its ring slot takes slice z + 1 from the
      // staging area; then the staging area takes slice z + 2 while slice z is worked on
      tc05::cp_async_wait_all();
      __syncthreads();
      if (z + 1 < S) stage_to_ring<N>(ring + ((z + 1) & 1) * SLOT, stg, beta);
      __syncthreads();
      if (z + 1 < z1 && z + 2 < S) stage_issue<N>(stg, x, xp, (size_t)(z + 2) * N2, r0, c0);
      float2 acc[kParts];
#pragma unroll
      for (int j = 0; j < kParts; ++j) acc[j] = f2(0.f);
      const size_t img = (size_t)z * N2 + acol;
      const bool more = z + 1 < z1;
      auto fin = [&](int t, float2 gsum, float2 yv) {
        const size_t ro = (size_t)(r0 + t) * N;
        const float2* v = fin_in + 3 * t * GP::THREADS;
        const float2 zd = v[0], at = v[GP::THREADS];
        const float2 Gv = f2fma(lam, gsum, f2fma(at, f2(-1.f), zd));
        acc[0] = f2fma(yv, zd, acc[0]);
        acc[1] = f2fma(yv, at, acc[1]);
        acc[4] = f2fma(Gv, Gv, acc[4]);
        if constexpr (MODE == (int)Pass3Mode::Gradient) {
          *reinterpret_cast<float2*>(out + img + ro) = Gv;
        } else if constexpr (UPDATE) {
          const float2 xv = v[2 * GP::THREADS];
          float2 xn = f2fma(f2(-invL), Gv, yv);
          if (pc.nonneg) xn = make_float2(fmaxf(xn.x, 0.f), fmaxf(xn.y, 0.f));
          *reinterpret_cast<float2*>(out + img + ro) = xn;
          acc[3] = f2fma(Gv, f2fma(xv, f2(-1.f), xn), acc[3]);
        }
        if (more) fetch(z + 1, t);  // this row's slots are free again
      };
      const float* s0 = ring + (z & 1) * SLOT;
      const float* s1 = ring + ((z + 1) & 1) * SLOT;
      if (rowe)
        band_step<N, Q2, PHI, false, true, true>(s0, s1, z + 1 < S, r0, c0w, ia, okL, okR, cr, edge, pk, pw, ph, fin);
      else if (cole)
        band_step<N, Q2, PHI, false, false, true>(s0, s1, z + 1 < S, r0, c0w, ia, okL, okR, cr, edge, pk, pw, ph,
                                                  fin);
      else
        band_step<N, Q2, PHI, false, false, false>(s0, s1, z + 1 < S, r0, c0w, ia, okL, okR, cr, edge, pk, pw, ph,
                                                   fin);
      if constexpr (PHI) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          acc[2] = f2fma(f2(wcls[j]), ph[j], acc[2]);
          ph[j] = f2(0.f);
        }
      }
#pragma unroll
      for (int j = 0; j < kParts; ++j) two_sum_add(hi[j], lo[j], acc[j].x + acc[j].y);
    }
  }
  block_partials_f<GP::WPB>(hi, lo, red, partials + (size_t)(block_offset + blockIdx.x) * kParts);
}

// ---------------------------------------------------------------- host launchers
template <int N>
static int set_smem_limits() {
  using Gm = Geo<N>;
  using Gr = Geo3a<N>;
  static bool done = false;
  if (done) return TMBIR_OK;
  if constexpr (N == 2048) {
    using Q = Q2048;
    const int s4 = (int)Q::sm_rows<4>(), s8 = (int)Q::sm_rows<8>();
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass1_q<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass1_q<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass1_q<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, s8));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass1_q<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, s8));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass2_q<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Q::SM2));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass2_q<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Q::SM2));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass3a_q<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass3a_q<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass3a_q<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, s8));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass3a_q<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, s8));
  } else if constexpr (is_block_fft_size<N>()) {
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
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass3a<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gr::SM1));
    TMBIR_CUDA(cudaFuncSetAttribute(k_pass3a<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gr::SM1));
  }
#define TMBIR_P3ATTR(M, Q)                                                                           \
  TMBIR_CUDA(cudaFuncSetAttribute(k_pass3<N, M, Q, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)GeoP<N>::SM));
  TMBIR_P3ATTR(0, true) TMBIR_P3ATTR(1, true) TMBIR_P3ATTR(2, true) TMBIR_P3ATTR(3, true) TMBIR_P3ATTR(4, true)
  TMBIR_P3ATTR(0, false) TMBIR_P3ATTR(1, false) TMBIR_P3ATTR(2, false) TMBIR_P3ATTR(3, false) TMBIR_P3ATTR(4, false)
#undef TMBIR_P3ATTR
  TMBIR_CUDA(cudaFuncSetAttribute(k_pass3<N, 3, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)GeoP<N>::SM));
  TMBIR_CUDA(cudaFuncSetAttribute(k_pass3<N, 3, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)GeoP<N>::SM));
  done = true;
  return TMBIR_OK;
}

// A group set of n groups, with each group's share of the launch's blocks.
template <class BlocksOf>
static GroupSet make_set(const GroupDev* gs, int n, BlocksOf&& blocks_of) {
  static_assert(sizeof(GroupSet) <= 4000, "group set exceeds the kernel parameter space");
  GroupSet set{};
  set.n = n;
  for (int i = 0; i < n; ++i) {
    set.g[i] = gs[i];
    set.boff[i + 1] = set.boff[i] + blocks_of(gs[i]);
  }
  return set;
}

template <int N>
static int pass1_n(const GroupDev* gs, int n, const StepArgs& a, bool bf16, cudaStream_t s) {
  using Gm = Geo<N>;
  if (int e = set_smem_limits<N>()) return e;
  if constexpr (N == 2048) {
    using Q = Q2048;
    if ((gs[0].rb1 ? gs[0].rb1 : Q::RB1) == 8) {
      const GroupSet set = make_set(gs, n, [](const GroupDev& g) { return g.S * (N / 8); });
      if (bf16)
        k_pass1_q<true, 8><<<set.boff[n], 512, Q::sm_rows<8>(), s>>>(set, a);
      else
        k_pass1_q<false, 8><<<set.boff[n], 512, Q::sm_rows<8>(), s>>>(set, a);
    } else {
      const GroupSet set = make_set(gs, n, [](const GroupDev& g) { return g.S * (N / 4); });
      if (bf16)
        k_pass1_q<true, 4><<<set.boff[n], 256, Q::sm_rows<4>(), s>>>(set, a);
      else
        k_pass1_q<false, 4><<<set.boff[n], 256, Q::sm_rows<4>(), s>>>(set, a);
    }
  } else if constexpr (is_block_fft_size<N>()) {
    using BG = BGeo<N>;
    const GroupSet set = make_set(gs, n, [](const GroupDev& g) { return g.S * BG::NB; });
    if (bf16)
      k_pass1_b<N, true><<<set.boff[n], BG::THREADS, BG::SM_ROWS, s>>>(set, a);
    else
      k_pass1_b<N, false><<<set.boff[n], BG::THREADS, BG::SM_ROWS, s>>>(set, a);
  } else {
    const GroupSet set = make_set(gs, n, [](const GroupDev& g) { return g.S * Gm::NB; });
    if (bf16)
      k_pass1<N, true><<<set.boff[n], Gm::THREADS, Gm::SM1, s>>>(set, a);
    else
      k_pass1<N, false><<<set.boff[n], Gm::THREADS, Gm::SM1, s>>>(set, a);
  }
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
template <int N>
static int pass2_n(const GroupDev* gs, int n, const IterState* st, bool bf16, cudaStream_t s) {
  using Gm = Geo<N>;
  if (int e = set_smem_limits<N>()) return e;
  if constexpr (N == 2048) {
    const GroupSet set = make_set(gs, n, [](const GroupDev& g) { return g.S * (N + 1); });
    if (bf16)
      k_pass2_q<true><<<set.boff[n], 128, Q2048::SM2, s>>>(set, st);
    else
      k_pass2_q<false><<<set.boff[n], 128, Q2048::SM2, s>>>(set, st);
  } else if constexpr (is_block_fft_size<N>()) {
    using BG = BGeo<N>;
    const GroupSet set = make_set(gs, n, [](const GroupDev& g) { return g.S * (N + 1); });
    if (bf16)
      k_pass2_b<N, true><<<set.boff[n], BG::THREADS, BG::SM_COL, s>>>(set, st);
    else
      k_pass2_b<N, false><<<set.boff[n], BG::THREADS, BG::SM_COL, s>>>(set, st);
  } else {
    const GroupSet set =
        make_set(gs, n, [](const GroupDev& g) { return (g.S * (N + 1) + Gm::CPB - 1) / Gm::CPB; });
    if (bf16)
      k_pass2<N, true><<<set.boff[n], Gm::THREADS, Gm::SM2, s>>>(set, st);
    else
      k_pass2<N, false><<<set.boff[n], Gm::THREADS, Gm::SM2, s>>>(set, st);
  }
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
template <int N, int MODE>
static int pass3_nm(const GroupDev* gs, int n, const StepArgs& a, const PriorC& pc, const float* apply_out,
                    int phase, double* partials, int off, cudaStream_t s) {
  using GP = GeoP<N>;
  static_assert(GP::NB * GP::CB == pass3_row_blocks(N), "pass-3b block count");
  // each group's slices per block resolved (tuned value or the default rule)
  GroupDev rz[kMergeMax];
  for (int i = 0; i < n; ++i) {
    rz[i] = gs[i];
    rz[i].zc = pass3_zc(gs[i], GP::NB * GP::CB);
  }
  const GroupSet set =
      make_set(rz, n, [](const GroupDev& g) { return GP::NB * GP::CB * ((pass3_slices(g) + g.zc - 1) / g.zc); });
  // a set of several groups only in Iterate mode (the other modes run one group per launch)
  if constexpr (MODE == 3) {
    if (n > 1) {
      if (pc.q_is_2)
        k_pass3<N, 3, true, true><<<set.boff[n], GP::THREADS, GP::SM, s>>>(set, a, pc, apply_out, phase, partials, off);
      else
        k_pass3<N, 3, false, true><<<set.boff[n], GP::THREADS, GP::SM, s>>>(set, a, pc, apply_out, phase, partials,
                                                                           off);
      TMBIR_CHECK_LAUNCH();
      return TMBIR_OK;
    }
  }
  if (n != 1) return set_error(TMBIR_ERR_ARG, "pass 3b takes several groups in Iterate mode only");
  if (pc.q_is_2 || MODE == 0)
    k_pass3<N, MODE, true, false><<<set.boff[n], GP::THREADS, GP::SM, s>>>(set, a, pc, apply_out, phase, partials, off);
  else
    k_pass3<N, MODE, false, false><<<set.boff[n], GP::THREADS, GP::SM, s>>>(set, a, pc, apply_out, phase, partials,
                                                                            off);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
// part: 1 pass 3a only, 2 pass 3b only, 3 both
template <int N>
static int pass3_n(const GroupDev* gs, int n, const StepArgs& a, Pass3Mode m, const PriorC& pc, double* partials,
                   int off, bool bf16, int part, cudaStream_t s) {
  using Gm = Geo3a<N>;
  if (int e = set_smem_limits<N>()) return e;
  if (n < 1 || n > kMergeMax) return set_error(TMBIR_ERR_ARG, "group set size");
  if (bf16 && m != Pass3Mode::Iterate) return set_error(TMBIR_ERR_ARG, "BF16 spectra are an iteration option only");
  // Apply writes K (*) x straight into the output; every other mode into the group's buffer
  float* apply_out = m == Pass3Mode::Apply ? a.out : nullptr;
  const IterState* st = m == Pass3Mode::Iterate ? a.st : nullptr;
  if (part & 1) {
    if constexpr (N == 2048) {
      using Q = Q2048;
      if ((gs[0].rb3 ? gs[0].rb3 : Q::RB3) == 8) {
        const GroupSet set = make_set(gs, n, [](const GroupDev& g) { return g.S * (N / 8); });
        if (bf16)
          k_pass3a_q<true, 8><<<set.boff[n], 512, Q::sm_rows<8>(), s>>>(set, st, apply_out);
        else
          k_pass3a_q<false, 8><<<set.boff[n], 512, Q::sm_rows<8>(), s>>>(set, st, apply_out);
      } else {
        const GroupSet set = make_set(gs, n, [](const GroupDev& g) { return g.S * (N / 4); });
        if (bf16)
          k_pass3a_q<true, 4><<<set.boff[n], 256, Q::sm_rows<4>(), s>>>(set, st, apply_out);
        else
          k_pass3a_q<false, 4><<<set.boff[n], 256, Q::sm_rows<4>(), s>>>(set, st, apply_out);
      }
    } else if constexpr (is_block_fft_size<N>()) {
      using BG = BGeo<N>;
      const GroupSet set = make_set(gs, n, [](const GroupDev& g) { return g.S * BG::NB; });
      if (bf16)
        k_pass3a_b<N, true><<<set.boff[n], BG::THREADS, BG::SM_ROWS, s>>>(set, st, apply_out);
      else
        k_pass3a_b<N, false><<<set.boff[n], BG::THREADS, BG::SM_ROWS, s>>>(set, st, apply_out);
    } else {
      const GroupSet set = make_set(gs, n, [](const GroupDev& g) { return g.S * Gm::NB; });
      if (bf16)
        k_pass3a<N, true><<<set.boff[n], Gm::THREADS, Gm::SM1, s>>>(set, st, apply_out);
      else
        k_pass3a<N, false><<<set.boff[n], Gm::THREADS, Gm::SM1, s>>>(set, st, apply_out);
    }
    TMBIR_CHECK_LAUNCH();
  }
  if (!(part & 2)) return TMBIR_OK;
  const int phase = bf16 ? 1 : 0;
  switch (m) {
    case Pass3Mode::Apply: return pass3_nm<N, 0>(gs, n, a, pc, apply_out, phase, partials, off, s);
    case Pass3Mode::Gradient: return pass3_nm<N, 1>(gs, n, a, pc, apply_out, phase, partials, off, s);
    case Pass3Mode::Step: return pass3_nm<N, 2>(gs, n, a, pc, apply_out, phase, partials, off, s);
    case Pass3Mode::Iterate: return pass3_nm<N, 3>(gs, n, a, pc, apply_out, phase, partials, off, s);
    default: return pass3_nm<N, 4>(gs, n, a, pc, apply_out, phase, partials, off, s);
  }
}

}  // namespace tmbir
