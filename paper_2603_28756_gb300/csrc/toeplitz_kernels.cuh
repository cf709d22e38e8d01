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

// rho'(d) (and rho(d) when PHI) of the qGGMRF potential
//   rho(d)  = |d/sigma|^q / (1 + u),            u = |d/(c sigma)|^(q-p)
//   rho'(d) = d/sigma^2 |d/sigma|^(q-2) (q + p u) / (1 + u)^2
template <bool Q2, bool PHI>
__device__ __forceinline__ float drho(float d, const PriorC& c, float& rho) {
  float a = fmaxf(fabsf(d), 1e-30f);
  float la = lg2a(a);
  float u = ex2a(c.qp * (la + lg2a(c.inv_csig)));
  float r = rcpa(1.0f + u);
  if constexpr (Q2) {
    if constexpr (PHI) rho = d * d * c.inv_sig2 * r;
    return d * c.inv_sig2 * fmaf(c.p, u, 2.0f) * r * r;
  } else {
    float aq2 = ex2a((c.q - 2.0f) * (la + lg2a(c.inv_sig)));
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
__device__ __forceinline__ void block_partials(float (&acc)[kParts], double* red, double* out) {
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kParts; ++j) {
    double v = warp_sum((double)acc[j]);
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
  const size_t base = ((size_t)(g.slice0 + s) * N + r) * N;

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
template <int N, int MODE, bool Q2>
__global__ void __launch_bounds__(Geo<N>::THREADS)
    k_pass3(GroupDev g, StepArgs a, PriorC pc, double* partials, int block_offset) {
  using Gm = Geo<N>;
  using F = typename Gm::F;
  constexpr int T = Gm::T, P = Gm::P, G = Gm::G, RB = Gm::RB, LD = Gm::LD;
  constexpr bool PRIOR = MODE != (int)Pass3Mode::Apply;
  constexpr bool PHI = MODE == (int)Pass3Mode::Step || MODE == (int)Pass3Mode::Iterate ||
                       MODE == (int)Pass3Mode::Objective;
  extern __shared__ float2 sm[];
  __shared__ double red[Gm::W * kParts];
  const float *x, *xp;
  float* out;
  float beta, invL;
  if constexpr (MODE == (int)Pass3Mode::Iterate) {
    if (a.st->done) return;
    const int cur = a.st->cur;
    x = a.xb[cur];
    xp = a.xb[(cur + 2) % 3];
    out = a.xb[(cur + 1) % 3];
    beta = (float)a.st->beta;
    invL = (float)a.st->invL;
  } else {
    x = a.x;
    xp = a.xprev;
    out = a.out;
    beta = a.beta;
    invL = a.invL;
  }
  const int s = blockIdx.x / Gm::NB, rb = blockIdx.x % Gm::NB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / T, t = lane % T;
  const int rl = warp * G + grp;
  const int r0 = rb * RB, r = r0 + rl;
  const size_t slice_base = (size_t)(g.slice0 + s) * N * N;
  const size_t base = slice_base + (size_t)r * N;

  // stage the half-spectrum rows of this block: tb[row][v]
  float2* tb = sm;
  {
    const float2* sp = g.spec + (size_t)s * (N + 1) * N + r0;
    for (int e = threadIdx.x; e < (N + 1) * RB; e += Gm::THREADS) {
      const int vv = e / RB, rr = e - vv * RB;
      tb[rr * LD + vv] = sp[(size_t)vv * N + rr];
    }
  }
  __syncthreads();
  // fold the Hermitian half spectrum into a packed length-N inverse transform:
  //   E[v] = Z[v] + conj(Z[N-v]),  O[v] = (Z[v] - conj(Z[N-v])) exp(+2 pi i v / 2N),  q = IFFT(E + iO)
  float2 q[P];
  SFor<0, P>::run([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const int vp = t + T * i;
    const float2 z = tb[rl * LD + vp];
    const float2 zr = tb[rl * LD + N - vp];
    const float2 e = make_float2(z.x + zr.x, z.y - zr.y);
    const float2 d = make_float2(z.x - zr.x, z.y + zr.y);
    const float2 o = cmulc(d, __ldg(&g.twM[vp]));
    q[i] = make_float2(e.x - o.y, e.y + o.x);
  });
  __syncthreads();
  F::template run<1>(q, sm + (warp * G + grp) * F::SMEM, g.twN, t);
  // q[i], i < P/2, holds (K(*)y)[r][2n], [r][2n+1] with n = t + T i

  float acc[kParts];
#pragma unroll
  for (int j = 0; j < kParts; ++j) acc[j] = 0.f;

  if constexpr (!PRIOR) {
    // operator only: z = K (*) x
    SFor<0, P / 2>::run([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      const int n = t + T * i;
      const float2 xv = __ldg(reinterpret_cast<const float2*>(x + base) + n);
      reinterpret_cast<float2*>(out + base)[n] = q[i];
      acc[0] += xv.x * q[i].x + xv.y * q[i].y;
      acc[5] += q[i].x * q[i].x + q[i].y * q[i].y;
    });
  } else {
    // y tile with one halo row and one halo slice on each side: yt[dz][row][col]
    __syncthreads();
    float* yt = reinterpret_cast<float*>(sm);
    constexpr int ROWS = RB + 2;
    for (int e = threadIdx.x; e < 3 * ROWS * (N / 4); e += Gm::THREADS) {
      const int c4 = e % (N / 4);
      const int rowi = (e / (N / 4)) % ROWS;
      const int dz = e / (ROWS * (N / 4));
      const int zz = s - 1 + dz, rr = r0 - 1 + rowi;
      float4 yv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (zz >= 0 && zz < g.S && rr >= 0 && rr < N) {
        const size_t off = ((size_t)(g.slice0 + zz) * N + rr) * N;
        const float4 xv = __ldg(reinterpret_cast<const float4*>(x + off) + c4);
        const float4 pv = __ldg(reinterpret_cast<const float4*>(xp + off) + c4);
        yv = make_float4(fmaf(beta, xv.x - pv.x, xv.x), fmaf(beta, xv.y - pv.y, xv.y),
                         fmaf(beta, xv.z - pv.z, xv.z), fmaf(beta, xv.w - pv.w, xv.w));
      }
      reinterpret_cast<float4*>(yt + (dz * ROWS + rowi) * N)[c4] = yv;
    }
    __syncthreads();
    const bool zval[3] = {s > 0, true, s + 1 < g.S};
    const bool rval[3] = {r > 0, true, r + 1 < N};
    const float wts[4] = {0.f, pc.wf, pc.we, pc.wc};
    SFor<0, P / 2>::run([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      const int n = t + T * i;
      const int c0 = 2 * n;
      const float* yc = yt + (1 * ROWS + rl + 1) * N;
      const float y0 = yc[c0], y1 = yc[c0 + 1];
      const float mL = c0 > 0 ? 1.f : 0.f, mR = c0 + 2 < N ? 1.f : 0.f;
      float g0 = 0.f, g1 = 0.f, ph = 0.f, rh = 0.f;
#pragma unroll
      for (int dz = 0; dz < 3; ++dz) {
        if (!zval[dz]) continue;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          if (!rval[dy]) continue;
          const float* rp = yt + (dz * ROWS + rl + dy) * N;
          const float A = rp[c0], B = rp[c0 + 1];
          const float Lf = c0 > 0 ? rp[c0 - 1] : 0.f;
          const float Rt = c0 + 2 < N ? rp[c0 + 2] : 0.f;
          const int ring = (dz != 1) + (dy != 1);
          const float w0 = wts[ring], w1 = wts[ring + 1];
          // forward offsets (lexicographic in dz, dy, dx) count each unordered pair once in Phi
          const bool fwd_plane = dz > 1 || (dz == 1 && dy > 1);
          if (ring != 0) {
            g0 += w0 * drho<Q2, PHI>(y0 - A, pc, rh);
            if (PHI && fwd_plane) ph += w0 * rh;
            g1 += w0 * drho<Q2, PHI>(y1 - B, pc, rh);
            if (PHI && fwd_plane) ph += w0 * rh;
            float f = w1 * drho<Q2, PHI>(y0 - B, pc, rh);  // (0, +1) from voxel 0
            g0 += f;
            if (PHI && fwd_plane) ph += w1 * rh;
            f = w1 * drho<Q2, PHI>(y1 - A, pc, rh);  // (0, -1) from voxel 1
            g1 += f;
            if (PHI && fwd_plane) ph += w1 * rh;
          } else {
            // the pair (voxel 0, voxel 1) itself: one evaluation, antisymmetric
            const float f = w1 * drho<Q2, PHI>(y0 - y1, pc, rh);
            g0 += f;
            g1 -= f;
            if (PHI) ph += w1 * rh;
          }
          g0 += mL * w1 * drho<Q2, PHI>(y0 - Lf, pc, rh);
          if (PHI && fwd_plane) ph += mL * w1 * rh;
          const float fr = mR * w1 * drho<Q2, PHI>(y1 - Rt, pc, rh);
          g1 += fr;
          if (PHI && (fwd_plane || ring == 0)) ph += mR * w1 * rh;
        }
      }
      const float2 zd = q[i];
      const float2 at = __ldg(reinterpret_cast<const float2*>(a.atg + base) + n);
      const float G0 = zd.x - at.x + pc.lam * g0;
      const float G1 = zd.y - at.y + pc.lam * g1;
      acc[0] += y0 * zd.x + y1 * zd.y;
      acc[1] += y0 * at.x + y1 * at.y;
      acc[2] += ph;
      acc[4] += G0 * G0 + G1 * G1;
      if constexpr (MODE == (int)Pass3Mode::Gradient) {
        reinterpret_cast<float2*>(out + base)[n] = make_float2(G0, G1);
      } else if constexpr (MODE == (int)Pass3Mode::Step || MODE == (int)Pass3Mode::Iterate) {
        const float2 xv = __ldg(reinterpret_cast<const float2*>(x + base) + n);
        const float n0 = fmaf(-invL, G0, y0), n1 = fmaf(-invL, G1, y1);
        reinterpret_cast<float2*>(out + base)[n] = make_float2(n0, n1);
        acc[3] += G0 * (n0 - xv.x) + G1 * (n1 - xv.y);
      }
    });
  }
  block_partials<Gm::W>(acc, red, partials + (size_t)(block_offset + blockIdx.x) * kParts);
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
                                  (int)Gm::SM3));
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
  if (pc.q_is_2 || MODE == 0)
    k_pass3<N, MODE, true><<<g.S * Gm::NB, Gm::THREADS, Gm::SM3, s>>>(g, a, pc, partials, off);
  else
    k_pass3<N, MODE, false><<<g.S * Gm::NB, Gm::THREADS, Gm::SM3, s>>>(g, a, pc, partials, off);
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
