// Register-resident DFT building blocks for the Toeplitz passes.
//
// A length-n FFT is computed by a group of T threads that each hold P = n / T
// complex values: thread t holds x[t + T*i], i = 0..P-1.  One transform is
//   stage A: a P-point DFT in registers over i, then the twiddle w_n^(t*k1);
//   exchange: a padded shared-memory transpose inside the warp;
//   stage B: T-point DFTs in registers over t.
// The result lands in the same distribution (thread t holds X[t + T*i]), so a
// forward transform, a point-wise multiply and an inverse transform need no
// reordering.  Small DFTs are fully unrolled at compile time with constant
// twiddles; trivial twiddles (multiples of pi/4) are strength-reduced.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>
#include <utility>

#include "dfloat.cuh"

namespace tmbir {

// ---------------------------------------------------------------- compile-time loops
template <int B, int E>
struct SFor {
  template <class F>
  __device__ __forceinline__ static void run(F&& f) {
    if constexpr (B < E) {
      f(std::integral_constant<int, B>{});
      SFor<B + 1, E>::run(f);
    }
  }
};

// ---------------------------------------------------------------- compile-time trig
// Taylor series on |x| <= pi/4 after exact rational octant reduction of 2*pi*k/n.
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double ct_sin_small(double x) {
  double t = x, s = x;
  for (int j = 1; j < 20; ++j) {
    t = -t * x * x / ((2.0 * j) * (2.0 * j + 1.0));
    s += t;
  }
  return s;
}
constexpr double ct_cos_small(double x) {
  double t = 1.0, s = 1.0;
  for (int j = 1; j < 20; ++j) {
    t = -t * x * x / ((2.0 * j - 1.0) * (2.0 * j));
    s += t;
  }
  return s;
}
// cos (which = 0) or sin (which = 1) of 2*pi*k/n: exact octant reduction with integers,
// then the series on an angle in [0, pi/4].
constexpr double ct_trig2pi(long long k, long long n, int which) {
  k %= n;
  if (k < 0) k += n;
  long long j = 8 * k;
  long long o = j / n, rem = j - o * n;
  double phi = (kPi / 4.0) * (double)rem / (double)n;        // angle within the octant
  double psi = (kPi / 4.0) * (double)(n - rem) / (double)n;  // pi/4 - phi
  double c = 0.0, s = 0.0;
  switch (o) {
    case 0: c = ct_cos_small(phi); s = ct_sin_small(phi); break;
    case 1: c = ct_sin_small(psi); s = ct_cos_small(psi); break;
    case 2: c = -ct_sin_small(phi); s = ct_cos_small(phi); break;
    case 3: c = -ct_cos_small(psi); s = ct_sin_small(psi); break;
    case 4: c = -ct_cos_small(phi); s = -ct_sin_small(phi); break;
    case 5: c = -ct_sin_small(psi); s = -ct_cos_small(psi); break;
    case 6: c = ct_sin_small(phi); s = -ct_cos_small(phi); break;
    default: c = ct_cos_small(psi); s = -ct_sin_small(psi); break;
  }
  return which == 0 ? c : s;
}

// ---------------------------------------------------------------- complex helpers
// Complex values are float2 (FP32 path) or double2 (FP64 setup path).
template <class C> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };
template <class C> using real_t = typename Real<C>::type;

__device__ __forceinline__ float2 mkc(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 mkc(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return fma(a, b, c); }
// double-word FP32 (the setup transforms of R*g): the same generic code, on the FP32 pipe
template <> struct Real<dfc> { using type = df; };
__device__ __forceinline__ dfc mkc(df x, df y) { return dfc{x, y}; }
__device__ __forceinline__ df fmar(df a, df b, df c) { return a * b + c; }

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
// FP32: one packed instruction for both parts (sm_100 and later), rounded like the scalar form
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  return mkc(fmar(a.x, b.x, -a.y * b.y), fmar(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <class C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mkc(fmar(a.x, b.x, a.y * b.y), fmar(a.y, b.x, -a.x * b.y));
}
template <class C> __device__ __forceinline__ C cconj(C a) { return mkc(a.x, -a.y); }
template <class C> __device__ __forceinline__ C cscale(C a, real_t<C> s) { return mkc(a.x * s, a.y * s); }
// a * (DIR * i)
template <int DIR, class C>
__device__ __forceinline__ C mul_diri(C a) {
  return DIR > 0 ? mkc(-a.y, a.x) : mkc(a.y, -a.x);
}
// twiddle: a * exp(DIR * 2*pi*i * K / N), K and N known at compile time
template <int K, int N, int DIR, class C>
__device__ __forceinline__ C twmul(C a) {
  using S = real_t<C>;
  constexpr int k = ((K % N) + N) % N;
  constexpr S r2 = (S)0.70710678118654752440084436210484904;
  if constexpr (k == 0) {
    return a;
  } else if constexpr (2 * k == N) {
    return mkc(-a.x, -a.y);
  } else if constexpr (4 * k == N) {
    return mul_diri<DIR>(a);
  } else if constexpr (4 * k == 3 * N) {
    return mul_diri<-DIR>(a);
  } else if constexpr (8 * k == N || 8 * k == 3 * N || 8 * k == 5 * N || 8 * k == 7 * N) {
    // (cs + i*ss) / sqrt(2) with cs, ss in {+1,-1}
    constexpr S cs = (8 * k == N || 8 * k == 7 * N) ? 1 : -1;
    constexpr S ss0 = (8 * k == N || 8 * k == 3 * N) ? 1 : -1;
    constexpr S ss = DIR > 0 ? ss0 : -ss0;
    return mkc(r2 * (cs * a.x - ss * a.y), r2 * (ss * a.x + cs * a.y));
  } else {
    constexpr S c = (S)ct_trig2pi(k, N, 0);
    constexpr S s = (S)(DIR * ct_trig2pi(k, N, 1));
    return mkc(fmar(a.x, c, -a.y * s), fmar(a.x, s, a.y * c));
  }
}

// ---------------------------------------------------------------- small DFTs, natural order in place
template <int P, int DIR, class C>
__device__ __forceinline__ void reg_dft(C (&a)[P]);

template <int DIR, class C>
__device__ __forceinline__ void dft2(C (&a)[2]) {
  C t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}
template <int DIR, class C>
__device__ __forceinline__ void dft4(C (&a)[4]) {
  C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  C t2 = cadd(a[1], a[3]), t3 = mul_diri<DIR>(csub(a[1], a[3]));
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = cadd(t1, t3);
  a[3] = csub(t1, t3);
}
template <int DIR, class C>
__device__ __forceinline__ void dft3(C (&a)[3]) {
  using S = real_t<C>;
  constexpr S h = (S)0.86602540378443864676372317075293618;  // sqrt(3)/2
  C t1 = cadd(a[1], a[2]), t2 = csub(a[1], a[2]);
  C x0 = cadd(a[0], t1);
  C m1 = mkc(fmar((S)-0.5, t1.x, a[0].x), fmar((S)-0.5, t1.y, a[0].y));
  C m2 = mul_diri<DIR>(mkc(h * t2.x, h * t2.y));
  a[0] = x0;
  a[1] = cadd(m1, m2);
  a[2] = csub(m1, m2);
}
template <int DIR, class C>
__device__ __forceinline__ void dft5(C (&a)[5]) {
  using S = real_t<C>;
  constexpr S c1 = (S)ct_trig2pi(1, 5, 0), c2 = (S)ct_trig2pi(2, 5, 0);
  constexpr S s1 = (S)ct_trig2pi(1, 5, 1), s2 = (S)ct_trig2pi(2, 5, 1);
  C t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
  C t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
  C x0 = cadd(a[0], cadd(t1, t2));
  C b1 = mkc(fmar(c1, t1.x, fmar(c2, t2.x, a[0].x)), fmar(c1, t1.y, fmar(c2, t2.y, a[0].y)));
  C b2 = mkc(fmar(c2, t1.x, fmar(c1, t2.x, a[0].x)), fmar(c2, t1.y, fmar(c1, t2.y, a[0].y)));
  C d1 = mul_diri<DIR>(mkc(fmar(s1, t3.x, s2 * t4.x), fmar(s1, t3.y, s2 * t4.y)));
  C d2 = mul_diri<DIR>(mkc(fmar(s2, t3.x, -s1 * t4.x), fmar(s2, t3.y, -s1 * t4.y)));
  a[0] = x0;
  a[1] = cadd(b1, d1);
  a[4] = csub(b1, d1);
  a[2] = cadd(b2, d2);
  a[3] = csub(b2, d2);
}

// Decimation in time: P = R * Q; X[k0 + Q*k1] = sum_r w_P^(r*k0) w_R^(r*k1) DFT_Q(x[r + R*q])[k0].
template <int P, int DIR, class C>
__device__ __forceinline__ void reg_dft(C (&a)[P]) {
  if constexpr (P == 1) {
  } else if constexpr (P == 2) {
    dft2<DIR>(a);
  } else if constexpr (P == 3) {
    dft3<DIR>(a);
  } else if constexpr (P == 4) {
    dft4<DIR>(a);
  } else if constexpr (P == 5) {
    dft5<DIR>(a);
  } else {
    constexpr int R = (P % 4 == 0) ? 4 : (P % 2 == 0 ? 2 : (P % 3 == 0 ? 3 : 5));
    constexpr int Q = P / R;
    static_assert(R * Q == P, "radix");
    C s[R][Q];
    SFor<0, R>::run([&](auto r_) {
      constexpr int r = decltype(r_)::value;
      SFor<0, Q>::run([&](auto q_) {
        constexpr int q = decltype(q_)::value;
        s[r][q] = a[r + R * q];
      });
      reg_dft<Q, DIR, C>(s[r]);
    });
    SFor<0, Q>::run([&](auto k0_) {
      constexpr int k0 = decltype(k0_)::value;
      C t[R];
      SFor<0, R>::run([&](auto r_) {
        constexpr int r = decltype(r_)::value;
        t[r] = twmul<r * k0, P, DIR>(s[r][k0]);
      });
      reg_dft<R, DIR, C>(t);
      SFor<0, R>::run([&](auto k1_) {
        constexpr int k1 = decltype(k1_)::value;
        a[k0 + Q * k1] = t[k1];
      });
    });
  }
}

// ---------------------------------------------------------------- group FFT of length n = T * P
// Thread layout in and out: thread t of the group holds x[t + T*i], i < P.
// tw: table of exp(-2*pi*i*t*k1/n) at tw[k1 * TWS * T + t] (conjugated on the fly for the
// inverse); TWS = 1 is the table [P][T] of this length, TWS = 2 reads every other row of the
// table of a transform twice as long (exp(-2 pi i t (2 k1) / 2n) = exp(-2 pi i t k1 / n)).
// sm: T*(P+1) complex values of shared memory owned by this group.
template <int T_, int P_>
struct GroupFFT {
  static constexpr int T = T_;
  static constexpr int P = P_;
  static constexpr int n = T * P;
  static constexpr int SMEM = T * (P + 1);  // complex elements
  static_assert(P % T == 0, "P must be a multiple of T");
  static_assert(T <= 32 && (32 % T) == 0, "group must divide a warp");

  template <int DIR, class C, int TWS = 1>
  __device__ __forceinline__ static void run(C (&v)[P], C* sm, const C* __restrict__ tw, int t) {
    reg_dft<P, DIR, C>(v);
    SFor<1, P>::run([&](auto k_) {
      constexpr int k1 = decltype(k_)::value;
      C w = __ldg(&tw[k1 * TWS * T + t]);
      v[k1] = DIR < 0 ? cmul(v[k1], w) : cmulc(v[k1], w);
    });
    __syncwarp();
    SFor<0, P>::run([&](auto k_) {
      constexpr int k1 = decltype(k_)::value;
      sm[t * (P + 1) + k1] = v[k1];
    });
    __syncwarp();
    constexpr int NB = P / T;
    SFor<0, NB>::run([&](auto m_) {
      constexpr int m = decltype(m_)::value;
      C b[T];
      SFor<0, T>::run([&](auto u_) {
        constexpr int u = decltype(u_)::value;
        b[u] = sm[u * (P + 1) + t + T * m];
      });
      reg_dft<T, DIR, C>(b);
      SFor<0, T>::run([&](auto k2_) {
        constexpr int k2 = decltype(k2_)::value;
        v[m + NB * k2] = b[k2];
      });
    });
  }
};

// group shape for a transform of length n (a power of two from 64 to 2048, or 1536, 2560)
template <int n>
struct FFTShape;
template <> struct FFTShape<64> { using type = GroupFFT<8, 8>; };
template <> struct FFTShape<128> { using type = GroupFFT<8, 16>; };
template <> struct FFTShape<256> { using type = GroupFFT<16, 16>; };
template <> struct FFTShape<512> { using type = GroupFFT<16, 32>; };
template <> struct FFTShape<1024> { using type = GroupFFT<32, 32>; };
template <> struct FFTShape<2048> { using type = GroupFFT<32, 64>; };
// Sides with a factor 3 or 5 use the block FFT (block_fft.cuh); the shape only fixes the rows
// per block of the row passes and of the stencil (32 threads per row).
template <int T_, int P_>
struct RowShape {
  static constexpr int T = T_, P = P_, SMEM = T * (P + 1);
};
template <> struct FFTShape<1536> { using type = RowShape<32, 48>; };
template <> struct FFTShape<2560> { using type = RowShape<32, 80>; };

}  // namespace tmbir
