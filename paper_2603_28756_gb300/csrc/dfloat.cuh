// Double-word FP32 arithmetic for the setup transforms of R*g.
//
// A value is hi + lo, two FP32 numbers with |lo| <= ulp(hi) / 2: a 48-bit significand, so each
// operation is accurate to about 2^-44 of its operands' magnitude (FP64 carries 2^-53).  The
// transforms that use it (the NUFFT adjoint of Eq. 4: the sparse gather onto the spreading grid,
// the 2D grid FFT, the deconvolution) then run on the FP32 pipe, whose rate on GB300 is
// sixty-four times the FP64 pipe's; their result is stored in FP32, whose 2^-24 is far above the
// double-word error even after the deconvolution's amplification (about 5e5 at the image
// corners on the 1.25x grid).
//
// The building blocks are the error-free transformations of floating-point arithmetic: Knuth's
// TwoSum (the exact rounding error of a sum), Dekker's FastTwoSum (the same when |a| >= |b|) and
// the FMA-based TwoProduct (the exact rounding error of a product, fma(a, b, -ab)).  The sum of
// two double-words is the "sloppy" form (TwoSum of the high parts, the low parts added, one
// renormalisation): its error is bounded relative to the operands' magnitudes, not to the
// result's, which is the bound an FFT or a dot product needs (their errors are judged against
// the input's norm).  Every step uses the _rn intrinsics, which the compiler never contracts
// into FMAs, so the transformations stay error-free.
#pragma once
#include <cuda_runtime.h>

namespace tmbir {

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // the double-word nearest to d: d rounded to FP32, then the remainder rounded to FP32
  __host__ __device__ constexpr df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr df(float f) : hi(f), lo(0.f) {}
  __host__ __device__ constexpr df(int i) : df((double)i) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ df operator+(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__host__ __device__ constexpr df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = __fmaf_rn(x.hi, y.hi, -p);  // the exact rounding error of hi * hi
  const float t = __fmaf_rn(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
  return fast_two_sum(p, __fadd_rn(e, t));
}

// a complex double-word, laid out like double2 (16 bytes, 16-byte aligned)
struct __align__(16) dfc {
  df x, y;
};

}  // namespace tmbir
