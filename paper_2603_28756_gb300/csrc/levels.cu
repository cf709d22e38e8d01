// Level transfer of the hierarchical reconstruction (Sec. 2.3): the x2 Lanczos-3 upsampler
// (Eqs. 16-17) and the coarse projections obtained by subsampling the detector.
#include "internal.h"

namespace tmbir {

// Lanczos kernel L(x) = sinc(x) sinc(x/3) at the half-integer offsets 2.5, 1.5, 0.5, -0.5,
// -1.5, -2.5 (the printed Eq. 16 is garbled; this is the standard windowed sinc), normalised to
// sum 1.  Filled on the host in FP64 and passed by value.
struct Lz3 {
  float w[6];
};

static Lz3 lanczos3_half_weights() {
  Lz3 z{};
  double w[6], s = 0.0;
  for (int t = 0; t < 6; ++t) {
    const double x = 2.5 - t;
    w[t] = 3.0 * std::sin(M_PI * x) * std::sin(M_PI * x / 3.0) / (M_PI * M_PI * x * x);
    s += w[t];
  }
  for (int t = 0; t < 6; ++t) z.w[t] = (float)(w[t] / s);
  return z;
}

// Separable x2 upsampling of one coarse row block per thread block:
//   pass over x into shared memory (coarse rows r0-2 .. r0+rows+2), then over y into the output.
// Fine sample 2i copies coarse sample i; fine sample 2i+1 = sum_t w[t] coarse[i-2+t].
__global__ void __launch_bounds__(256) k_upsample(const float* __restrict__ in, int S, int Nc, float* __restrict__ out, Lz3 z) {
  extern __shared__ float tmp[];  // [(RB + 5)][2 Nc]
  const int RB = 8;
  const int Nf = 2 * Nc;
  const int blocks_per_slice = (Nc + RB - 1) / RB;
  const int s = blockIdx.x / blocks_per_slice, rb = blockIdx.x % blocks_per_slice;
  const int r0 = rb * RB;
  const float* src = in + (size_t)s * Nc * Nc;
  // x pass for coarse rows r0-2 .. r0+RB+2 (zero outside)
  const int rows = RB + 5;
  for (int e = threadIdx.x; e < rows * Nf; e += blockDim.x) {
    const int j = e % Nf, lr = e / Nf, r = r0 - 2 + lr;
    float v = 0.f;
    if (r >= 0 && r < Nc) {
      const float* row = src + (size_t)r * Nc;
      const int i = j >> 1;
      if ((j & 1) == 0) {
        v = row[i];
      } else {
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          const int i2 = i - 2 + t;
          if (i2 >= 0 && i2 < Nc) v = fmaf(z.w[t], row[i2], v);
        }
      }
    }
    tmp[lr * Nf + j] = v;
  }
  __syncthreads();
  // y pass: fine rows 2 r0 .. 2 (r0 + RB) - 1
  float* dst = out + (size_t)s * Nf * Nf;
  for (int e = threadIdx.x; e < 2 * RB * Nf; e += blockDim.x) {
    const int j = e % Nf, fr = 2 * r0 + e / Nf;
    if (fr >= Nf) continue;
    const int i = fr >> 1;
    float v;
    if ((fr & 1) == 0) {
      v = tmp[(i - r0 + 2) * Nf + j];
    } else {
      v = 0.f;
#pragma unroll
      for (int t = 0; t < 6; ++t) v = fmaf(z.w[t], tmp[(i - 2 + t - r0 + 2) * Nf + j], v);
    }
    dst[(size_t)fr * Nf + j] = v;
  }
}

int launch_upsample_lanczos3(const float* in, int S, int Nc, float* out, cudaStream_t s) {
  const Lz3 z = lanczos3_half_weights();
  const int RB = 8;
  const size_t smem = (size_t)(RB + 5) * 2 * Nc * sizeof(float);
  if (smem > 200 * 1024) return set_error(TMBIR_ERR_SHAPE, "upsample: coarse grid too wide");
  static bool attr = false;
  if (!attr) {
    TMBIR_CUDA(cudaFuncSetAttribute(k_upsample, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  const int blocks = S * ((Nc + RB - 1) / RB);
  k_upsample<<<blocks, 256, smem, s>>>(in, S, Nc, out, z);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

__global__ void k_downsample(const float* __restrict__ in, size_t rows, int nd, int f, float* __restrict__ out) {
  const int ndc = nd / f;
  const float inv = 1.0f / (float)f;
  const size_t total = rows * ndc;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const size_t row = id / ndc;
    const int m = (int)(id % ndc);
    out[id] = in[row * nd + (size_t)f * m] * inv;
  }
}

int launch_downsample_sino(const float* in, int S, int na, int nd, int f, float* out, cudaStream_t s) {
  const size_t rows = (size_t)S * na;
  const size_t total = rows * (nd / f);
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 32);
  k_downsample<<<blocks, 256, 0, s>>>(in, rows, nd, f, out);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

}  // namespace tmbir
