// Block-wide mixed-radix FFT in shared memory (Stockham autosort, FP32) for the image sides
// whose padded transforms are not powers of two: 1536 = 2^9 * 3 and 2560 = 2^9 * 5.  All threads
// of the block take part; a stage with radix R gives each thread n / R R-point DFTs in
// registers (the same small DFTs as the group FFT), with twiddles from a plain table
// tw[j] = exp(-2 pi i j / n).  Natural order in and out.
#pragma once
#include "fft.cuh"

namespace tmbir {

// radix plan per transform length (the Stockham recursion takes the radices in any order)
template <int n>
struct BlockPlan;
template <>
struct BlockPlan<1536> {
  static constexpr int NS = 4;
  static constexpr int R[NS] = {8, 8, 8, 3};
};
template <>
struct BlockPlan<2560> {
  static constexpr int NS = 4;
  static constexpr int R[NS] = {8, 8, 8, 5};
};

template <int n>
constexpr bool is_block_fft_size() {
  return n == 1536 || n == 2560;
}

// one Stockham stage: Y[(j - k) R + k + m Ls] = DFT_R over m of X[j + m n/R] w^(k m n/(Ls R)),
// k = j mod Ls (k m n/(Ls R) < n, so the table index needs no reduction)
template <int R, int DIR>
__device__ __forceinline__ void block_stage(const float2* X, float2* Y, int n, int Ls, const float2* __restrict__ tw) {
  const int nb = n / R;
  const int tstep = n / (Ls * R);
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int k = j % Ls;
    float2 a[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      float2 v = X[j + m * nb];
      if (m > 0 && k > 0) {
        const float2 w = __ldg(&tw[k * m * tstep]);
        v = DIR < 0 ? cmul(v, w) : cmulc(v, w);
      }
      a[m] = v;
    }
    reg_dft<R, DIR, float2>(a);
    const int o = (j - k) * R + k;
#pragma unroll
    for (int m = 0; m < R; ++m) Y[o + m * Ls] = a[m];
  }
}

// Transform of X (n complex, shared memory) using Y as the second buffer; returns the buffer
// that holds the result.  Starts and ends with a barrier of the whole block.
template <int n, int DIR>
__device__ __forceinline__ float2* block_fft(float2* X, float2* Y, const float2* __restrict__ tw) {
  using PL = BlockPlan<n>;
  __syncthreads();
  float2* src = X;
  float2* dst = Y;
  int Ls = 1;
  SFor<0, PL::NS>::run([&](auto s_) {
    constexpr int s = decltype(s_)::value;
    constexpr int R = PL::R[s];
    block_stage<R, DIR>(src, dst, n, Ls, tw);
    __syncthreads();
    Ls *= R;
    float2* t = src;
    src = dst;
    dst = t;
  });
  return src;
}

}  // namespace tmbir
