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
#pragma once
#include "fft.cuh"
#include "internal.h"

namespace tmbir {

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

// rho'(d) (and rho(d) when PHI) of the qGGMRF potential
//   rho(d)  = |d/sigma|^q / (1 + u),            u = |d/(c sigma)|^(q-p)
//   rho'(d) = d/sigma^2 |d/sigma|^(q-2) (q + p u) / (1 + u)^2
// Two special-function operations (log2 and exp2) per call; the reciprocal runs on the FMA pipe.
template <bool Q2, bool PHI>
__device__ __forceinline__ float drho(float d, const PriorC& c, float& rho) {
  const float a = fmaxf(fabsf(d), 1e-30f);
  const float la = lg2a(a);
  const float u = ex2a(fmaf(c.qp, la, c.qp * c.l2_inv_csig));
  const float r = rcp_newton(1.0f + u);
  if constexpr (Q2) {
    if constexpr (PHI) rho = d * d * c.inv_sig2 * r;
    return d * c.inv_sig2 * fmaf(c.p, u, 2.0f) * r * r;
  } else {
    const float aq2 = ex2a((c.q - 2.0f) * (la + c.l2_inv_sig));
    if constexpr (PHI) rho = aq2 * d * d * c.inv_sig2 * r;
    return d * c.inv_sig2 * aq2 * fmaf(c.p, u, c.q) * r * r;
  }
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
template <int N>
__global__ void __launch_bounds__(Geo<N>::THREADS) k_pass1(GroupDev g, StepArgs a) {
  using Gm = Geo<N>;
  using F = typename Gm::F;
  constexpr int T = Gm::T, P = Gm::P, G = Gm::G, RB = Gm::RB, LD = Gm::LD;
  extern __shared__ float2 sm[];
  const float *x, *xp;
  float beta;
  if (a.st) {
    if (a.st->done) return;
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
  float2* out = g.spec + (size_t)s * (N + 1) * N + rb * RB;
  for (int e = threadIdx.x; e < (N + 1) * RB; e += Gm::THREADS) {
    const int vv = e / RB, rr = e - vv * RB;
    out[(size_t)vv * N + rr] = tb[rr * LD + vv];
  }
}

// ---------------------------------------------------------------- pass 2: columns
template <int N>
__global__ void __launch_bounds__(Geo<N>::THREADS) k_pass2(GroupDev g, const IterState* st) {
  using Gm = Geo<N>;
  using F = typename Gm::F;
  constexpr int T = Gm::T, P = Gm::P, G = Gm::G;
  extern __shared__ float2 sm[];
  if (st && st->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / T, t = lane % T;
  const int unit = warp * G + grp, h = unit & 1;
  const int col = blockIdx.x * Gm::CPB + (unit >> 1);
  const int ncols = g.S * (N + 1);
  const bool active = col < ncols;
  const int vcol = active ? col / g.S : 0, s = active ? col % g.S : 0;  // slices fastest: kernel column reuse
  float2* p = g.spec + ((size_t)s * (N + 1) + vcol) * N;
  float2 v[P];
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const int rr = t + T * i;
    float2 w = active ? p[rr] : make_float2(0.f, 0.f);
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
      p[rr] = cadd(v[i], os[rr]);
    });
  }
}

// ---------------------------------------------------------------- pass 3: rows, inverse + gradient
// A block owns RB consecutive rows of one group and marches through a chunk of its slices.
// Per slice: the inverse row transforms give K (*) y for the block's rows; then the qGGMRF
// gradient is accumulated pair by pair.  For the neighbourhood, thread t owns a band of RS
// rows and KCH chunks of CHW columns.  A neighbour pair whose two voxels the same thread owns
// (in the same slice, or in consecutive slices of the block's chunk) is evaluated once and
// applied to both voxels -- the next-slice half is carried in registers to the next step;
// every other pair is evaluated from each side for that side only.  Each unordered pair
// enters Phi once, from the voxel it is a forward offset of (lexicographic in dz, dy, dx).
template <int N>
struct Geo3 {
  using Gm = Geo<N>;
  static constexpr int RB = Gm::RB, THREADS = Gm::THREADS;
  static constexpr int RS = 4;                      // rows per band
  static constexpr int NBAND = RB / RS;
  static constexpr int NSTRIP = THREADS / NBAND;    // column strips per band
  static constexpr int CW = N / NSTRIP;             // columns per thread
  static constexpr int CHW = CW < 4 ? CW : 4;       // columns per chunk
  static constexpr int KCH = CW / CHW;              // chunks per thread
  static constexpr int ROWS = RB + 2;               // ring rows (one halo row each side)
  static constexpr size_t SM_RING = (size_t)2 * ROWS * N * sizeof(float);
  static constexpr size_t SM_A = Gm::cmax(Gm::SM1, (size_t)RB * N * sizeof(float));
  static constexpr size_t SM = SM_A + SM_RING;
  static_assert(NBAND * RS == RB && NSTRIP * NBAND == THREADS && KCH * CHW * NSTRIP == N, "stencil layout");
};

// y = x + beta (x - x_prev) for block rows -1 .. RB of one slice into a ring slot (zero outside)
template <int N>
__device__ __forceinline__ void load_ring(float* slot, const float* x, const float* xp, float beta, size_t off_slice,
                                          int r0, bool valid_slice) {
  using G3 = Geo3<N>;
  for (int e = threadIdx.x; e < G3::ROWS * (N / 4); e += G3::THREADS) {
    const int c4 = e % (N / 4), rowi = e / (N / 4);
    const int rr = r0 - 1 + rowi;
    float4 yv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid_slice && rr >= 0 && rr < N) {
      const size_t off = off_slice + (size_t)rr * N;
      const float4 xv = __ldg(reinterpret_cast<const float4*>(x + off) + c4);
      const float4 pv = __ldg(reinterpret_cast<const float4*>(xp + off) + c4);
      yv = make_float4(fmaf(beta, xv.x - pv.x, xv.x), fmaf(beta, xv.y - pv.y, xv.y), fmaf(beta, xv.z - pv.z, xv.z),
                       fmaf(beta, xv.w - pv.w, xv.w));
    }
    reinterpret_cast<float4*>(slot + rowi * N)[c4] = yv;
  }
}

template <int N, int MODE, bool Q2>
__global__ void __launch_bounds__(Geo<N>::THREADS)
    k_pass3(GroupDev g, StepArgs a, PriorC pc, double* partials, int block_offset, int zc) {
  using Gm = Geo<N>;
  using G3 = Geo3<N>;
  using F = typename Gm::F;
  constexpr int T = Gm::T, P = Gm::P, G = Gm::G, RB = Gm::RB, LD = Gm::LD;
  constexpr int RS = G3::RS, CHW = G3::CHW, KCH = G3::KCH, NSTRIP = G3::NSTRIP, ROWS = G3::ROWS;
  constexpr bool PRIOR = MODE != (int)Pass3Mode::Apply;
  constexpr bool PHI = MODE == (int)Pass3Mode::Step || MODE == (int)Pass3Mode::Iterate ||
                       MODE == (int)Pass3Mode::Objective;
  constexpr bool UPDATE = MODE == (int)Pass3Mode::Step || MODE == (int)Pass3Mode::Iterate;
  extern __shared__ float2 sm[];
  __shared__ double red[Gm::W * kParts];
  const float *x, *xp;
  float* out;
  float beta, invL;
  if constexpr (MODE == (int)Pass3Mode::Iterate) {
    if (a.st->done) return;
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
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / T, t = lane % T;
  const int rl = warp * G + grp;
  const int r0 = rb * RB;
  // stencil ownership
  const int band = threadIdx.x / NSTRIP, strip = threadIdx.x % NSTRIP;
  const int brow0 = band * RS;  // first block row of the band
  float2* tb = sm;
  float* kzs = reinterpret_cast<float*>(sm);  // K(*)y of the block rows, [RB][N], after the transforms
  float* ring = reinterpret_cast<float*>(reinterpret_cast<char*>(sm) + G3::SM_A);
  const size_t N2 = (size_t)N * N;

  double dacc[kParts];
#pragma unroll
  for (int j = 0; j < kParts; ++j) dacc[j] = 0.0;
  float own[RS][KCH * CHW], nxt[RS][KCH * CHW];
#pragma unroll
  for (int i = 0; i < RS; ++i)
#pragma unroll
    for (int j = 0; j < KCH * CHW; ++j) own[i][j] = nxt[i][j] = 0.f;

  if constexpr (PRIOR) {
    load_ring<N>(ring + (z0 & 1) * ROWS * N, x, xp, beta, g.img_off + (size_t)z0 * N2, r0, true);
    if (z0 > 0) load_ring<N>(ring + ((z0 - 1) & 1) * ROWS * N, x, xp, beta, g.img_off + (size_t)(z0 - 1) * N2, r0, true);
  }
  const float wts[4] = {0.f, pc.wf, pc.we, pc.wc};
  const float mL = (strip == 0) ? 0.f : 1.f;           // chunk 0's left halo column exists
  const float mR = (strip == NSTRIP - 1) ? 0.f : 1.f;  // last chunk's right halo column exists

  for (int z = z0; z < z1; ++z) {
    const size_t slice_base = g.img_off + (size_t)z * N2;
    // ---- K (*) y for rows r0 .. r0+RB-1 of slice z
    __syncthreads();
    {
      const float2* sp = g.spec + (size_t)z * (N + 1) * N + r0;
      for (int e = threadIdx.x; e < (N + 1) * RB; e += Gm::THREADS) {
        const int vv = e / RB, rr = e - vv * RB;
        tb[rr * LD + vv] = sp[(size_t)vv * N + rr];
      }
    }
    __syncthreads();
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
    __syncthreads();
    SFor<0, P / 2>::run([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      reinterpret_cast<float2*>(kzs + rl * N)[t + T * i] = q[i];
    });

    float yo[RS][KCH * CHW];  // own y values of slice z
    float acc[kParts];
#pragma unroll
    for (int j = 0; j < kParts; ++j) acc[j] = 0.f;

    if constexpr (PRIOR) {
      const float* slot_z = ring + (z & 1) * ROWS * N;
      SFor<0, RS>::run([&](auto i_) {
        constexpr int i = decltype(i_)::value;
        SFor<0, KCH>::run([&](auto k_) {
          constexpr int k = decltype(k_)::value;
          const int col0 = CHW * (strip + NSTRIP * k);
          SFor<0, CHW>::run([&](auto c_) {
            constexpr int ci = decltype(c_)::value;
            yo[i][k * CHW + ci] = slot_z[(brow0 + i + 1) * N + col0 + ci];
          });
        });
      });
      // pair evaluation against one partner row (slice z + DZ, band row PR), for every own row
      // within one row of it.  SHARED: the partner slice is processed by this block (both ends
      // owned by one thread are then updated here, or were already, see below).
      auto pairs = [&](auto dz_, auto pr_, const float* slot, bool shared_z) {
        constexpr int DZ = decltype(dz_)::value, PR = decltype(pr_)::value;
        float pv[KCH][CHW + 2];
        const int prow = brow0 + PR;  // partner block row
        SFor<0, KCH>::run([&](auto k_) {
          constexpr int k = decltype(k_)::value;
          const int col0 = CHW * (strip + NSTRIP * k);
          const float* rp = slot + (prow + 1) * N;
          SFor<0, CHW>::run([&](auto c_) {
            constexpr int ci = decltype(c_)::value;
            pv[k][ci + 1] = rp[col0 + ci];
          });
          pv[k][0] = rp[col0 > 0 ? col0 - 1 : 0];
          pv[k][CHW + 1] = rp[col0 + CHW < N ? col0 + CHW : N - 1];
        });
        SFor<0, RS>::run([&](auto i_) {
          constexpr int RR = decltype(i_)::value;
          constexpr int DY = PR - RR;
          if constexpr (DY >= -1 && DY <= 1) {
            SFor<0, KCH>::run([&](auto k_) {
              constexpr int k = decltype(k_)::value;
              SFor<0, CHW>::run([&](auto c_) {
                constexpr int ci = decltype(c_)::value;
                SFor<0, 3>::run([&](auto d_) {
                  constexpr int DX = decltype(d_)::value - 1;
                  if constexpr (!(DZ == 0 && DY == 0 && DX == 0)) {
                    constexpr bool owned = PR >= 0 && PR < RS && ci + DX >= 0 && ci + DX < CHW;
                    constexpr bool fwd = DZ > 0 || (DZ == 0 && (DY > 0 || (DY == 0 && DX > 0)));
                    constexpr int ring_n = (DZ != 0) + (DY != 0) + (DX != 0);
                    // 0: skip, 1: both ends (same slice), 2: own end (+ next-slice end if shared)
                    constexpr int kind = DZ == 0 ? (owned ? (fwd ? 1 : 0) : 2) : (DZ > 0 ? 2 : (owned ? 3 : 2));
                    if constexpr (kind != 0) {
                      // kind 3: owned partner in slice z-1, evaluated at step z-1 unless z is the chunk start
                      if (kind != 3 || !shared_z) {
                        float m = 1.f;
                        if constexpr (ci + DX < 0) m = (k == 0) ? mL : 1.f;
                        if constexpr (ci + DX >= CHW) m = (k == KCH - 1) ? mR : 1.f;
                        const float w = wts[ring_n];
                        float rh = 0.f;
                        const float f = w * drho<Q2, PHI>(yo[RR][k * CHW + ci] - pv[k][ci + DX + 1], pc, rh);
                        if constexpr (kind == 1) {
                          own[RR][k * CHW + ci] += f;
                          own[PR][k * CHW + ci + DX] -= f;
                          if constexpr (PHI) acc[2] += w * rh;
                        } else {
                          own[RR][k * CHW + ci] += m * f;
                          if constexpr (PHI && fwd) acc[2] += m * w * rh;
                          if constexpr (DZ > 0 && owned) {
                            if (shared_z) nxt[PR][k * CHW + ci + DX] -= f;
                          }
                        }
                      }
                    }
                  }
                });
              });
            });
          }
        });
      };
      const bool row_lo = r0 + brow0 - 1 >= 0, row_hi = r0 + brow0 + RS < N;
      // slice z - 1 (own end only, except owned pairs at the chunk start)
      if (z > 0) {
        const float* slot_m = ring + ((z - 1) & 1) * ROWS * N;
        const bool shared_m = z - 1 >= z0;
        if (row_lo) pairs(std::integral_constant<int, -1>{}, std::integral_constant<int, -1>{}, slot_m, shared_m);
        SFor<0, RS>::run([&](auto p_) { pairs(std::integral_constant<int, -1>{}, p_, slot_m, shared_m); });
        if (row_hi) pairs(std::integral_constant<int, -1>{}, std::integral_constant<int, RS>{}, slot_m, shared_m);
      }
      __syncthreads();  // kzs complete; slot of z - 1 free
      if (z + 1 < g.S)
        load_ring<N>(ring + ((z + 1) & 1) * ROWS * N, x, xp, beta, slice_base + N2, r0, true);
      __syncthreads();
      // slice z
      if (row_lo) pairs(std::integral_constant<int, 0>{}, std::integral_constant<int, -1>{}, slot_z, true);
      SFor<0, RS>::run([&](auto p_) { pairs(std::integral_constant<int, 0>{}, p_, slot_z, true); });
      if (row_hi) pairs(std::integral_constant<int, 0>{}, std::integral_constant<int, RS>{}, slot_z, true);
      // slice z + 1
      if (z + 1 < g.S) {
        const float* slot_p = ring + ((z + 1) & 1) * ROWS * N;
        const bool shared_p = z + 1 < z1;
        if (row_lo) pairs(std::integral_constant<int, 1>{}, std::integral_constant<int, -1>{}, slot_p, shared_p);
        SFor<0, RS>::run([&](auto p_) { pairs(std::integral_constant<int, 1>{}, p_, slot_p, shared_p); });
        if (row_hi) pairs(std::integral_constant<int, 1>{}, std::integral_constant<int, RS>{}, slot_p, shared_p);
      }
    } else {
      __syncthreads();
    }

    // ---- per voxel: gradient, update, partial sums (CHW consecutive columns at a time)
    SFor<0, RS>::run([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      const int row = r0 + brow0 + i;
      const size_t rbase = slice_base + (size_t)row * N;
      SFor<0, KCH>::run([&](auto k_) {
        constexpr int k = decltype(k_)::value;
        const int col0 = CHW * (strip + NSTRIP * k);
        float zd[CHW], at[CHW], xv[CHW], res[CHW];
        (void)res;
        SFor<0, CHW>::run([&](auto c_) {
          constexpr int ci = decltype(c_)::value;
          zd[ci] = kzs[(brow0 + i) * N + col0 + ci];
        });
        const bool need_x = !PRIOR || UPDATE;
        const bool need_at = PRIOR;
        if constexpr (CHW == 4) {
          if (need_x) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(x + rbase + col0));
            xv[0] = v.x; xv[1] = v.y; xv[2] = v.z; xv[3] = v.w;
          }
          if (need_at) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(a.atg + rbase + col0));
            at[0] = v.x; at[1] = v.y; at[2] = v.z; at[3] = v.w;
          }
        } else {
          SFor<0, CHW>::run([&](auto c_) {
            constexpr int ci = decltype(c_)::value;
            if (need_x) xv[ci] = __ldg(x + rbase + col0 + ci);
            if (need_at) at[ci] = __ldg(a.atg + rbase + col0 + ci);
          });
        }
        SFor<0, CHW>::run([&](auto c_) {
          constexpr int ci = decltype(c_)::value;
          if constexpr (!PRIOR) {
            res[ci] = zd[ci];
            acc[0] += xv[ci] * zd[ci];
            acc[5] += zd[ci] * zd[ci];
          } else {
            const float yv = yo[i][k * CHW + ci];
            const float Gv = zd[ci] - at[ci] + pc.lam * own[i][k * CHW + ci];
            acc[0] += yv * zd[ci];
            acc[1] += yv * at[ci];
            acc[4] += Gv * Gv;
            if constexpr (MODE == (int)Pass3Mode::Gradient) {
              res[ci] = Gv;
            } else if constexpr (UPDATE) {
              const float xn = fmaf(-invL, Gv, yv);
              res[ci] = xn;
              acc[3] += Gv * (xn - xv[ci]);
            }
          }
        });
        if constexpr (MODE != (int)Pass3Mode::Objective) {
          if constexpr (CHW == 4) {
            *reinterpret_cast<float4*>(out + rbase + col0) = make_float4(res[0], res[1], res[2], res[3]);
          } else {
            SFor<0, CHW>::run([&](auto c_) {
              constexpr int ci = decltype(c_)::value;
              out[rbase + col0 + ci] = res[ci];
            });
          }
        }
      });
    });
#pragma unroll
    for (int j = 0; j < kParts; ++j) dacc[j] += (double)acc[j];
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
      for (int j = 0; j < KCH * CHW; ++j) {
        own[i][j] = nxt[i][j];
        nxt[i][j] = 0.f;
      }
  }
  block_partials<Gm::W>(dacc, red, partials + (size_t)(block_offset + blockIdx.x) * kParts);
}

// ---------------------------------------------------------------- host launchers
template <int N>
static int set_smem_limits() {
  using Gm = Geo<N>;
  static bool done = false;
  if (done) return TMBIR_OK;
  TMBIR_CUDA(cudaFuncSetAttribute(k_pass1<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::SM1));
  TMBIR_CUDA(cudaFuncSetAttribute(k_pass2<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::SM2));
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
static int pass1_n(const GroupDev& g, const StepArgs& a, cudaStream_t s) {
  using Gm = Geo<N>;
  if (int e = set_smem_limits<N>()) return e;
  k_pass1<N><<<g.S * Gm::NB, Gm::THREADS, Gm::SM1, s>>>(g, a);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
template <int N>
static int pass2_n(const GroupDev& g, const IterState* st, cudaStream_t s) {
  using Gm = Geo<N>;
  if (int e = set_smem_limits<N>()) return e;
  const int blocks = (g.S * (N + 1) + Gm::CPB - 1) / Gm::CPB;
  k_pass2<N><<<blocks, Gm::THREADS, Gm::SM2, s>>>(g, st);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
template <int N, int MODE>
static int pass3_nm(const GroupDev& g, const StepArgs& a, const PriorC& pc, double* partials, int off,
                    cudaStream_t s) {
  using Gm = Geo<N>;
  if (int e = set_smem_limits<N>()) return e;
  const int zc = pass3_slices_per_block(g.S, Gm::NB);
  const int blocks = Gm::NB * ((g.S + zc - 1) / zc);
  if (pc.q_is_2 || MODE == 0)
    k_pass3<N, MODE, true><<<blocks, Gm::THREADS, Geo3<N>::SM, s>>>(g, a, pc, partials, off, zc);
  else
    k_pass3<N, MODE, false><<<blocks, Gm::THREADS, Geo3<N>::SM, s>>>(g, a, pc, partials, off, zc);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
template <int N>
static int pass3_n(const GroupDev& g, const StepArgs& a, Pass3Mode m, const PriorC& pc, double* partials, int off,
                   cudaStream_t s) {
  switch (m) {
    case Pass3Mode::Apply: return pass3_nm<N, 0>(g, a, pc, partials, off, s);
    case Pass3Mode::Gradient: return pass3_nm<N, 1>(g, a, pc, partials, off, s);
    case Pass3Mode::Step: return pass3_nm<N, 2>(g, a, pc, partials, off, s);
    case Pass3Mode::Iterate: return pass3_nm<N, 3>(g, a, pc, partials, off, s);
    default: return pass3_nm<N, 4>(g, a, pc, partials, off, s);
  }
}

}  // namespace tmbir
