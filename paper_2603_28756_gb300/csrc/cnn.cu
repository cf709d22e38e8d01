// Learned warm start: a four-layer 3x3 convolutional refiner (1 -> 32 -> 32 -> 32 -> 1, ReLU
// after the first three layers, zero padding) applied to the normalised FBP start, with its
// own training kernels.  The paper has no learned component; this refiner is an addition.
//
// Precision: FP32 master weights, BF16 activations and weight copies, FP32 accumulation.
// The two 32 -> 32 layers are implicit GEMMs on the 5th-generation tensor cores (tcgen05.mma,
// BF16 operands in shared memory, FP32 accumulators in TMEM): M = 128 pixels of an image row,
// N = 32 output channels, K = 9 taps x 32 channels.
// Their data gradient is the same kernel run on the flipped, transposed weights.  The first
// and last layers (32 MACs per tap) and all weight gradients run on the CUDA cores; weight
// gradients are reduced over a fixed set of blocks in a fixed order (deterministic).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "internal.h"
#include "tc05.cuh"

namespace tmbir {

constexpr int kC = 32;                          // channels of the hidden layers
constexpr int kW0 = kC * 9, kB0 = kC;           // layer 0: [co][tap], bias
constexpr int kW1 = kC * kC * 9, kB1 = kC;      // layers 1, 2: [co][ci][tap] (oracle layout)
constexpr int kW3 = kC * 9, kB3 = 1;            // layer 3: [ci][tap]
constexpr int kOff0 = 0, kOffB0 = kW0;
constexpr int kOff1 = kOffB0 + kB0, kOffB1 = kOff1 + kW1;
constexpr int kOff2 = kOffB1 + kB1, kOffB2 = kOff2 + kW1;
constexpr int kOff3 = kOffB2 + kB1, kOffB3 = kOff3 + kW3;
constexpr int kParams = kOffB3 + kB3;  // 19105
constexpr int kTM = 128;               // pixels of one tensor-core tile (MMA M): a run of one image row
constexpr int kTX = kTM + 2;           // staged pixels of a row: x0 - 1 .. x0 + kTM
constexpr int kChunkB = kTX * 16;      // bytes of one staged (row, 8-channel chunk) array
constexpr int kRows = 4;                          // output rows of one tile (independent accumulators)
constexpr int kStageA = (kRows + 2) * 4 * kChunkB;  // staged rows x four chunks
constexpr int kStageAPad = (kStageA + 127) / 128 * 128;
constexpr int kWElems = 9 * 4 * kC * 8;           // packed 32 -> 32 weights [tap][chunk][n][8]
constexpr int kConvSmem = kStageAPad + kWElems * 2;  // staged rows + weights
constexpr uint32_t kMmaPolls = 1u << 22;          // bound of every wait on an MMA completion
constexpr int kWgradBlocks = 304;      // blocks of the weight-gradient reductions

struct CnnNet {
  cudaStream_t stream;
  int max_batch, H, W;
  float* master;        // [kParams] FP32 weights (oracle layout)
  float* grad;          // [kParams]
  float* adam_m;        // [kParams]
  float* adam_v;        // [kParams]
  __nv_bfloat16* wg1;   // layer 1 as the MMA's B operand: [tap][k chunk][co][8], k = ci
  __nv_bfloat16* wg2;   // layer 2
  __nv_bfloat16* wt1;   // flipped transpose of layer 1 for the data gradient: [tap][k chunk][ci][8], k = co
  __nv_bfloat16* wt2;
  int* err;             // set when a bounded wait on the tensor core gives up
  __nv_bfloat16* a0;    // activations NHWC [B][H][W][32]
  __nv_bfloat16* a1;
  __nv_bfloat16* a2;
  __nv_bfloat16* g1;    // gradients NHWC
  __nv_bfloat16* g2;
  float* xin;           // [B][H][W] normalised input
  float* out;           // [B][H][W] network output
  float* gout;          // [B][H][W]
  float* sig;           // [B] per-image scale
  float* wpart;         // [kWgradBlocks][kW1] weight-gradient partials
  double* dpart;        // scalar partials
  int step;
};

// ---------------------------------------------------------------- weight layouts
// Weights of the two 32 -> 32 layers in the layout of the MMA's B operand (no swizzle,
// K-major): element (tap, k chunk j, row n, e) = W[n][k = 8 j + e][tap] for the forward pass and
// the flipped transpose W[co = 8 j + e][ci = n][8 - tap] for the data gradient.
__global__ void k_cnn_pack(const float* __restrict__ master, __nv_bfloat16* wg1, __nv_bfloat16* wg2,
                           __nv_bfloat16* wt1, __nv_bfloat16* wt2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kWElems; i += gridDim.x * blockDim.x) {
    const int e = i % 8, n = (i / 8) % kC, j = (i / (8 * kC)) % 4, tap = i / (32 * kC);
    const int k = 8 * j + e;
    wg1[i] = __float2bfloat16_rn(master[kOff1 + (n * kC + k) * 9 + tap]);
    wg2[i] = __float2bfloat16_rn(master[kOff2 + (n * kC + k) * 9 + tap]);
    wt1[i] = __float2bfloat16_rn(master[kOff1 + (k * kC + n) * 9 + (8 - tap)]);
    wt2[i] = __float2bfloat16_rn(master[kOff2 + (k * kC + n) * 9 + (8 - tap)]);
  }
}

// ---------------------------------------------------------------- tensor-core 32 -> 32 convolution
// out[p][n] = sum_{tap, c} w[tap][n][c] in[p + tap][c] (+ bias, ReLU), as an implicit GEMM on the
// 5th-generation tensor cores.  A tile is kRows image rows x 128 pixels; each of its rows is an
// MMA with M = 128 pixels and N = 32 output channels, and each of the nine taps is one K = 32
// step (two K = 16 MMAs).  The kRows accumulators (32 TMEM columns each) are independent, and
// the MMAs are issued tap-major across them so consecutive MMAs do not wait on one another.
// The input rows y0-1 .. y0+kRows (pixels x0-1..x0+128, zero outside the image) are staged
// once per tile as 8-channel chunks, [row][chunk][pixel][8], which is the no-swizzle K-major
// operand layout; tap (dy, dx) of output row r is staged row r + dy started dx pixels (16
// bytes) later.  Each warp moves its 32 pixels of every row out with tcgen05.ld.
// MASK (data gradient): the result is multiplied by (mask[p][n] > 0).
template <bool BIAS_RELU, bool MASK>
__global__ void __launch_bounds__(128) k_conv32(const __nv_bfloat16* __restrict__ in, int B, int H, int W,
                                                const __nv_bfloat16* __restrict__ wpk, const float* __restrict__ bias,
                                                const __nv_bfloat16* __restrict__ mask, __nv_bfloat16* __restrict__ out,
                                                int* err) {
  namespace tc = tc05;
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* sa = smraw;
  unsigned char* sw = smraw + kStageAPad;
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t IDESC = tc::idesc_bf16_f32<kTM, kC>();
  const unsigned char* wsrc = reinterpret_cast<const unsigned char*>(wpk);
  for (int i = threadIdx.x; i < kWElems * 2 / 16; i += blockDim.x) tc::cp_async16(sw + 16 * i, wsrc + 16 * i, true);
  if (warp == 0) tc::tmem_alloc<kRows * kC>(&tmem_base);
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t a_base = tc::smem_addr(sa), w_base = tc::smem_addr(sw);
  const uint64_t a_desc = tc::smem_desc(a_base, kChunkB, 128), w_desc = tc::smem_desc(w_base, kC * 16, 128);
  float bias_r[kC];
#pragma unroll
  for (int c = 0; c < kC; ++c) bias_r[c] = BIAS_RELU ? __ldg(bias + c) : 0.f;
  const int tiles_x = (W + kTM - 1) / kTM, tiles_y = (H + kRows - 1) / kRows;
  const int ntiles = B * tiles_y * tiles_x;
  uint32_t parity = 0;
  bool failed = false;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, b = tile / (tiles_x * tiles_y);
    const int y0 = ty * kRows, x0 = tx * kTM;
    // thread t copies staged pixel t (threads 0, 1 also pixels 128, 129) of every staged row
    for (int px = threadIdx.x; px < kTX; px += blockDim.x) {
      const int gx = x0 - 1 + px;
      const bool vx = gx >= 0 && gx < W;
#pragma unroll
      for (int sr = 0; sr < kRows + 2; ++sr) {
        const int gy = y0 + sr - 1;
        const bool v = vx && gy >= 0 && gy < H;
        const __nv_bfloat16* src = v ? in + (((size_t)b * H + gy) * W + gx) * kC : in;
        unsigned char* dst = sa + sr * 4 * kChunkB + px * 16;
#pragma unroll
        for (int j = 0; j < 4; ++j) tc::cp_async16(dst + j * kChunkB, v ? src + 8 * j : in, v);
      }
    }
    tc::cp_async_wait_all();  // this tile's rows (and, the first time, the weights)
    tc::fence_async_shared();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      // every operand start is a fixed byte offset from the staging / weight bases, added to the
      // descriptors' start-address field (bytes >> 4; the offsets stay inside the 14-bit field)
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const uint64_t bd = w_desc + (uint64_t)(((tap * 4 + 2 * s) * (kC * 16)) >> 4);
#pragma unroll
          for (int r = 0; r < kRows; ++r) {
            const uint64_t ad = a_desc + (uint64_t)((((r + dy) * 4 + 2 * s) * kChunkB + dx * 16) >> 4);
            tc::mma_bf16(tmem + r * kC, ad, bd, IDESC, (tap | s) ? 1u : 0u);
          }
        }
      }
      tc::mma_commit(&bar);
    }
    const bool ok = tc::mbar_wait(&bar, parity, kMmaPolls);
    parity ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    const int gx = x0 + warp * 32 + lane;
#pragma unroll 1
    for (int r = 0; r < kRows; ++r) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + r * kC, v);
      const int gy = y0 + r;
      if (gx >= W || gy >= H) continue;
      const size_t pbase = (((size_t)b * H + gy) * W + gx) * kC;
      if constexpr (BIAS_RELU) {
#pragma unroll
        for (int c = 0; c < kC; ++c) v[c] = fmaxf(v[c] + bias_r[c], 0.f);
      }
      if constexpr (MASK) {
        const uint4* mk = reinterpret_cast<const uint4*>(mask + pbase);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 m = mk[q];
          const __nv_bfloat162* mb = reinterpret_cast<const __nv_bfloat162*>(&m);
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float2 f = __bfloat1622float2(mb[h]);
            if (!(f.x > 0.f)) v[8 * q + 2 * h] = 0.f;
            if (!(f.y > 0.f)) v[8 * q + 2 * h + 1] = 0.f;
          }
        }
      }
      uint4* dst = reinterpret_cast<uint4*>(out + pbase);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint4 o;
        __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
        for (int h = 0; h < 4; ++h) ob[h] = __floats2bfloat162_rn(v[8 * q + 2 * h], v[8 * q + 2 * h + 1]);
        dst[q] = o;
      }
    }
    // TMEM and the staged rows are reused by the next tile
    tc::fence_before_sync();
    __syncthreads();
  }
  if (failed) {
    // give the outstanding MMAs a second bounded chance to finish before freeing their TMEM
    tc::mbar_wait(&bar, parity ^ 1u, kMmaPolls);
    if (threadIdx.x == 0) atomicExch(err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc<kRows * kC>(tmem);
}

// ---------------------------------------------------------------- first and last layers (CUDA cores)
// a0[p][co] = relu(b0[co] + sum_tap w0[co][tap] x[p + tap]).  A block stages an 8 x 32 tile of
// x with a one-pixel halo; thread t owns output channels 4 (t % 8) .. +3 (weights in
// registers) for the pixels t / 8 + 32 k, so the eight threads of a pixel write its 64 bytes.
constexpr int kFH = 8, kFW = 32;
__global__ void __launch_bounds__(256) k_conv_first(const float* __restrict__ x, int B, int H, int W,
                                                    const float* __restrict__ master, __nv_bfloat16* __restrict__ a0) {
  __shared__ float xt[kFH + 2][kFW + 2];
  const int cg = threadIdx.x & 7, ps = threadIdx.x >> 3;
  float wr[4][9], br[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
#pragma unroll
    for (int t = 0; t < 9; ++t) wr[c][t] = master[kOff0 + (4 * cg + c) * 9 + t];
    br[c] = master[kOff0 + kW0 + 4 * cg + c];
  }
  const int tiles_x = (W + kFW - 1) / kFW, tiles_y = (H + kFH - 1) / kFH;
  const int tpi = tiles_x * tiles_y;
  for (int tile = blockIdx.x; tile < B * tpi; tile += gridDim.x) {
    const int b = tile / tpi, ty = (tile % tpi) / tiles_x, tx = tile % tiles_x;
    const int y0 = ty * kFH, x0 = tx * kFW;
    __syncthreads();
    for (int q = threadIdx.x; q < (kFH + 2) * (kFW + 2); q += blockDim.x) {
      const int gy = y0 - 1 + q / (kFW + 2), gx = x0 - 1 + q % (kFW + 2);
      xt[q / (kFW + 2)][q % (kFW + 2)] =
          (gy >= 0 && gy < H && gx >= 0 && gx < W) ? x[((size_t)b * H + gy) * W + gx] : 0.f;
    }
    __syncthreads();
#pragma unroll 2
    for (int ly = 0; ly < kFH; ++ly) {
      const int gy = y0 + ly, gx = x0 + ps;
      if (gy >= H || gx >= W) continue;
      float nb[9];
#pragma unroll
      for (int t = 0; t < 9; ++t) nb[t] = xt[ly + t / 3][ps + t % 3];
      float v[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float acc = br[c];
#pragma unroll
        for (int t = 0; t < 9; ++t) acc = fmaf(wr[c][t], nb[t], acc);
        v[c] = fmaxf(acc, 0.f);
      }
      uint2 o;
      reinterpret_cast<__nv_bfloat162*>(&o)[0] = __floats2bfloat162_rn(v[0], v[1]);
      reinterpret_cast<__nv_bfloat162*>(&o)[1] = __floats2bfloat162_rn(v[2], v[3]);
      *reinterpret_cast<uint2*>(a0 + (((size_t)b * H + gy) * W + gx) * kC + 4 * cg) = o;
    }
  }
}

// out[p] = b3 + sum_{tap, ci} w3[ci][tap] a2[p + tap][ci], as out[p] = b3 + sum_tap T[p + tap][tap]
// with T[q][tap] = sum_ci w3[ci][tap] a2[q][ci]: a block computes T once per pixel of its 8 x 32
// tile plus a one-pixel halo (each activation vector read once) and sums the nine shifted
// entries from shared memory.
constexpr int kLH = 8, kLW = 32;
__global__ void __launch_bounds__(256, 2) k_conv_last(const __nv_bfloat16* __restrict__ a2, int B, int H, int W,
                                                      const float* __restrict__ master, float* __restrict__ out) {
  __shared__ __align__(16) float w[kC][12];  // w3[ci][tap], rows padded to 12 for 16-byte vector reads
  __shared__ float T[(kLH + 2) * (kLW + 2)][9];
  for (int i = threadIdx.x; i < kC * 9; i += blockDim.x) w[i / 9][i % 9] = master[kOff3 + i];
  const float b3 = master[kOff3 + kW3];
  const int tiles_x = (W + kLW - 1) / kLW, tiles_y = (H + kLH - 1) / kLH;
  const int tpi = tiles_x * tiles_y;
  for (int tile = blockIdx.x; tile < B * tpi; tile += gridDim.x) {
    const int b = tile / tpi, ty = (tile % tpi) / tiles_x, tx = tile % tiles_x;
    const int y0 = ty * kLH, x0 = tx * kLW;
    __syncthreads();  // weights loaded; T of the previous tile consumed
    for (int q = threadIdx.x; q < (kLH + 2) * (kLW + 2); q += blockDim.x) {
      const int gy = y0 - 1 + q / (kLW + 2), gx = x0 - 1 + q % (kLW + 2);
      float t[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) t[k] = 0.f;
      if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
        const uint4* src = reinterpret_cast<const uint4*>(a2 + (((size_t)b * H + gy) * W + gx) * kC);
#pragma unroll 1
        for (int v4 = 0; v4 < 4; ++v4) {
          const uint4 u = src[v4];
          const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            const float a = h & 1 ? __high2float(h2[h / 2]) : __low2float(h2[h / 2]);
            const float* wr = w[8 * v4 + h];
            const float4 w0 = *reinterpret_cast<const float4*>(wr);
            const float4 w1 = *reinterpret_cast<const float4*>(wr + 4);
            t[0] = fmaf(w0.x, a, t[0]);
            t[1] = fmaf(w0.y, a, t[1]);
            t[2] = fmaf(w0.z, a, t[2]);
            t[3] = fmaf(w0.w, a, t[3]);
            t[4] = fmaf(w1.x, a, t[4]);
            t[5] = fmaf(w1.y, a, t[5]);
            t[6] = fmaf(w1.z, a, t[6]);
            t[7] = fmaf(w1.w, a, t[7]);
            t[8] = fmaf(wr[8], a, t[8]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) T[q][k] = t[k];
    }
    __syncthreads();
    const int ly = threadIdx.x / kLW, lx = threadIdx.x % kLW;
    const int gy = y0 + ly, gx = x0 + lx;
    if (gy < H && gx < W) {
      float s = b3;
#pragma unroll
      for (int k = 0; k < 9; ++k) s += T[(ly + k / 3) * (kLW + 2) + lx + k % 3][k];
      out[((size_t)b * H + gy) * W + gx] = s;
    }
  }
}

// g2[p][ci] = (a2[p][ci] > 0) * sum_tap w3[ci][tap] gout[p - tap]
__global__ void k_last_dgrad(const float* __restrict__ gout, const __nv_bfloat16* __restrict__ a2, int B, int H, int W,
                             const float* __restrict__ master, __nv_bfloat16* __restrict__ g2) {
  __shared__ float w[kW3];
  for (int i = threadIdx.x; i < kW3; i += blockDim.x) w[i] = master[kOff3 + i];
  __syncthreads();
  const size_t total = (size_t)B * H * W;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
    const int xx = (int)(p % W), yy = (int)((p / W) % H);
    const size_t b = p / ((size_t)H * W);
    float gg[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int gy = yy - (t / 3 - 1), gx = xx - (t % 3 - 1);
      gg[t] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? gout[(b * H + gy) * W + gx] : 0.f;
    }
    const __nv_bfloat162* a = reinterpret_cast<const __nv_bfloat162*>(a2 + p * kC);
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(g2 + p * kC);
#pragma unroll 4
    for (int c = 0; c < kC; c += 2) {
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        s0 = fmaf(w[c * 9 + t], gg[t], s0);
        s1 = fmaf(w[(c + 1) * 9 + t], gg[t], s1);
      }
      const float2 av = __bfloat1622float2(a[c / 2]);
      o[c / 2] = __floats2bfloat162_rn(av.x > 0.f ? s0 : 0.f, av.y > 0.f ? s1 : 0.f);
    }
  }
}

// ---------------------------------------------------------------- weight gradients (fixed-order block partials)
// Layer 1/2: dW[co][ci][tap] = sum_p g[p][co] in[p + tap][ci]; thread t owns co = t / 8 and
// ci = 4 (t % 8) .. +3 for all 9 taps (36 sums); pixels in a fixed grid-stride order.
__global__ void __launch_bounds__(256) k_wgrad32(const __nv_bfloat16* __restrict__ g, const __nv_bfloat16* __restrict__ in,
                                                 int B, int H, int W, float* __restrict__ part) {
  const int co = threadIdx.x >> 3, ci0 = (threadIdx.x & 7) * 4;
  float s[4][9];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int t = 0; t < 9; ++t) s[i][t] = 0.f;
  const size_t total = (size_t)B * H * W;
  for (size_t p = blockIdx.x; p < total; p += gridDim.x) {
    const int xx = (int)(p % W), yy = (int)((p / W) % H);
    const size_t b = p / ((size_t)H * W);
    const float gv = __bfloat162float(g[p * kC + co]);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int gy = yy + t / 3 - 1, gx = xx + t % 3 - 1;
      if (gy < 0 || gy >= H || gx < 0 || gx >= W) continue;
      const __nv_bfloat162* a = reinterpret_cast<const __nv_bfloat162*>(in + ((b * H + gy) * W + gx) * kC + ci0);
      const float2 v0 = __bfloat1622float2(a[0]), v1 = __bfloat1622float2(a[1]);
      s[0][t] = fmaf(gv, v0.x, s[0][t]);
      s[1][t] = fmaf(gv, v0.y, s[1][t]);
      s[2][t] = fmaf(gv, v1.x, s[2][t]);
      s[3][t] = fmaf(gv, v1.y, s[3][t]);
    }
  }
  float* o = part + (size_t)blockIdx.x * kW1;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int t = 0; t < 9; ++t) o[(co * kC + ci0 + i) * 9 + t] = s[i][t];
}

// Layer 0: dW0[co][tap] = sum_p g0[p][co] xin[p + tap], db0[co] = sum_p g0[p][co];
// thread t: co = t % 32, taps 3 (t / 32) .. +2 for t < 96, bias for 96 <= t < 128.
// Partial row layout: [0, 288) dW0, [288, 320) db0.
__global__ void __launch_bounds__(128) k_wgrad_first(const __nv_bfloat16* __restrict__ g0, const float* __restrict__ xin,
                                                     int B, int H, int W, float* __restrict__ part) {
  const int co = threadIdx.x & 31, role = threadIdx.x >> 5;
  float acc[3] = {0.f, 0.f, 0.f};
  const size_t total = (size_t)B * H * W;
  for (size_t p = blockIdx.x; p < total; p += gridDim.x) {
    const float gv = __bfloat162float(g0[p * kC + co]);
    if (role == 3) {
      acc[0] += gv;
      continue;
    }
    const int xx = (int)(p % W), yy = (int)((p / W) % H);
    const size_t b = p / ((size_t)H * W);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int t = role * 3 + j;
      const int gy = yy + t / 3 - 1, gx = xx + t % 3 - 1;
      if (gy >= 0 && gy < H && gx >= 0 && gx < W) acc[j] = fmaf(gv, xin[(b * H + gy) * W + gx], acc[j]);
    }
  }
  float* o = part + (size_t)blockIdx.x * kW1;
  if (role < 3) {
#pragma unroll
    for (int j = 0; j < 3; ++j) o[co * 9 + role * 3 + j] = acc[j];
  } else {
    o[288 + co] = acc[0];
  }
}
// Hidden-layer bias: db[co] = sum_p g[p][co]; partial row [0, 32)
__global__ void __launch_bounds__(32) k_bias_grad(const __nv_bfloat16* __restrict__ g, size_t total, float* __restrict__ part) {
  float acc = 0.f;
  for (size_t p = blockIdx.x; p < total; p += gridDim.x) acc += __bfloat162float(g[p * kC + threadIdx.x]);
  part[(size_t)blockIdx.x * kW1 + threadIdx.x] = acc;
}
// Layer 3: dW3[ci][tap] = sum_p gout[p] a2[p + tap][ci], db3 = sum_p gout[p];
// thread t < 32: ci = t, all taps; thread 32: bias.  Partial row [0, 288) dW3, [288] db3.
__global__ void __launch_bounds__(64) k_wgrad_last(const float* __restrict__ gout, const __nv_bfloat16* __restrict__ a2,
                                                   int B, int H, int W, float* __restrict__ part) {
  const int ci = threadIdx.x;
  float acc[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) acc[t] = 0.f;
  const size_t total = (size_t)B * H * W;
  for (size_t p = blockIdx.x; p < total; p += gridDim.x) {
    const float gv = gout[p];
    if (ci == 32) {
      acc[0] += gv;
      continue;
    }
    if (ci > 32) continue;
    const int xx = (int)(p % W), yy = (int)((p / W) % H);
    const size_t b = p / ((size_t)H * W);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int gy = yy + t / 3 - 1, gx = xx + t % 3 - 1;
      if (gy >= 0 && gy < H && gx >= 0 && gx < W)
        acc[t] = fmaf(gv, __bfloat162float(a2[((b * H + gy) * W + gx) * kC + ci]), acc[t]);
    }
  }
  float* o = part + (size_t)blockIdx.x * kW1;
  if (ci < 32) {
#pragma unroll
    for (int t = 0; t < 9; ++t) o[ci * 9 + t] = acc[t];
  } else if (ci == 32) {
    o[288] = acc[0];
  }
}
// gin[p] = sum_{tap, co} w0[co][tap] g0[p - tap][co]
__global__ void k_first_dgrad(const __nv_bfloat16* __restrict__ g0, int B, int H, int W, const float* __restrict__ master,
                              float* __restrict__ gin) {
  __shared__ float w[kW0];
  for (int i = threadIdx.x; i < kW0; i += blockDim.x) w[i] = master[kOff0 + i];
  __syncthreads();
  const size_t total = (size_t)B * H * W;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
    const int xx = (int)(p % W), yy = (int)((p / W) % H);
    const size_t b = p / ((size_t)H * W);
    float s = 0.f;
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
      const int gy = yy - (t / 3 - 1), gx = xx - (t % 3 - 1);
      if (gy < 0 || gy >= H || gx < 0 || gx >= W) continue;
      const __nv_bfloat162* gg = reinterpret_cast<const __nv_bfloat162*>(g0 + ((b * H + gy) * W + gx) * kC);
#pragma unroll
      for (int c = 0; c < kC; c += 2) {
        const float2 v = __bfloat1622float2(gg[c / 2]);
        s = fmaf(w[c * 9 + t], v.x, s);
        s = fmaf(w[(c + 1) * 9 + t], v.y, s);
      }
    }
    gin[p] = s;
  }
}
// dst[i] += sum over blocks (fixed order) of part[b][i], i < n
__global__ void k_reduce_parts(const float* __restrict__ part, int nblocks, int n, float* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * kW1 + i];
    dst[i] += (float)s;
  }
}

// ---------------------------------------------------------------- normalisation, loss, optimiser
// per image: sig = sqrt(mean x^2) (1 if zero); xin = x / sig.  kNormBlocks blocks per image
// each reduce a strided share in FP64, then one block per image adds the shares in order.
constexpr int kNormBlocks = 64;
__global__ void k_norm_partial(const float* __restrict__ x, int HW, double* __restrict__ part) {
  __shared__ double sh[256];
  const int b = blockIdx.y;
  const float* xb = x + (size_t)b * HW;
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += kNormBlocks * blockDim.x) s += (double)xb[i] * xb[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)b * kNormBlocks + blockIdx.x] = sh[0];
}
__global__ void k_norm_stats(const double* __restrict__ part, int HW, float* __restrict__ sig) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < kNormBlocks; ++k) s += part[(size_t)blockIdx.x * kNormBlocks + k];
  const double r = sqrt(s / HW);
  sig[blockIdx.x] = r > 0 ? (float)r : 1.f;
}
__global__ void k_scale_in(const float* __restrict__ x, int HW, size_t total, const float* __restrict__ sig,
                           float* __restrict__ xin) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    xin[i] = x[i] / sig[i / HW];
}
// refined = x + sig * net
__global__ void k_residual_out(const float* __restrict__ x, const float* __restrict__ net, int HW, size_t total,
                               const float* __restrict__ sig, float* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    y[i] = x[i] + sig[i / HW] * net[i];
}
// loss = mean (net - (t - x)/sig)^2; gout = 2 (net - r) / P; per-block FP64 partials
__global__ void k_loss(const float* __restrict__ net, const float* __restrict__ x, const float* __restrict__ t, int HW,
                       size_t total, const float* __restrict__ sig, float* __restrict__ gout, double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  const float inv = 1.0f / (float)total;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const float r = (t[i] - x[i]) / sig[i / HW];
    const float d = net[i] - r;
    gout[i] = 2.0f * d * inv;
    s += (double)d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void k_sum_d(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s * scale;
  }
}
// Adam (Kingma & Ba 2015) on the FP32 master weights
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ---------------------------------------------------------------- host sequences
static size_t cnn_bytes(int B, int H, int W, size_t* offs) {
  size_t off = 0;
  auto take = [&](size_t b) {
    off = (off + 255) / 256 * 256;
    size_t o = off;
    off += b;
    return o;
  };
  const size_t P = (size_t)B * H * W;
  offs[0] = take(kParams * 4);                         // master
  offs[1] = take(kParams * 4);                         // grad
  offs[2] = take(kParams * 4);                         // m
  offs[3] = take(kParams * 4);                         // v
  for (int i = 0; i < 4; ++i) offs[4 + i] = take((size_t)kWElems * 2);  // wg1 wg2 wt1 wt2
  for (int i = 0; i < 5; ++i) offs[8 + i] = take(P * kC * 2);           // a0 a1 a2 g1 g2
  for (int i = 0; i < 3; ++i) offs[13 + i] = take(P * 4);               // xin out gout
  offs[16] = take((size_t)B * 4);                                        // sig
  offs[17] = take((size_t)kWgradBlocks * kW1 * 4);                       // wpart
  offs[18] = take(std::max<size_t>(4096, (size_t)B * kNormBlocks) * 8);  // dpart (loss / norm partials)
  offs[19] = take(256);                                                  // err
  return (off + 255) / 256 * 256;
}

static int conv32(CnnNet& n, const __nv_bfloat16* in, int B, const __nv_bfloat16* w, const float* bias,
                  const __nv_bfloat16* mask, __nv_bfloat16* out, bool relu) {
  static bool attr = false;
  if (!attr) {
    TMBIR_CUDA(cudaFuncSetAttribute(k_conv32<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem));
    TMBIR_CUDA(cudaFuncSetAttribute(k_conv32<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem));
    attr = true;
  }
  const int tiles = B * ((n.H + kRows - 1) / kRows) * ((n.W + kTM - 1) / kTM);
  const int blocks = std::min(tiles, 152 * 3);
  if (relu)
    k_conv32<true, false><<<blocks, 128, kConvSmem, n.stream>>>(in, B, n.H, n.W, w, bias, nullptr, out, n.err);
  else
    k_conv32<false, true><<<blocks, 128, kConvSmem, n.stream>>>(in, B, n.H, n.W, w, bias, mask, out, n.err);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
// TMBIR_ERR_TIMEOUT (and the flag cleared) when a convolution gave up waiting on the tensor core;
// reads the flag after the stream has drained up to here
static int check_tc(CnnNet& n) {
  int flag = 0;
  TMBIR_CUDA(cudaMemcpyAsync(&flag, n.err, sizeof(int), cudaMemcpyDeviceToHost, n.stream));
  TMBIR_CUDA(cudaStreamSynchronize(n.stream));
  if (flag) {
    TMBIR_CUDA(cudaMemsetAsync(n.err, 0, sizeof(int), n.stream));
    return set_error(TMBIR_ERR_TIMEOUT, "cnn: a tensor-core convolution timed out waiting for its MMAs");
  }
  return TMBIR_OK;
}

static int net_forward(CnnNet& n, int B) {
  const size_t P = (size_t)B * n.H * n.W;
  const int blocks = (int)std::min<size_t>((P + 255) / 256, 152 * 16);
  k_conv_first<<<blocks, 256, 0, n.stream>>>(n.xin, B, n.H, n.W, n.master, n.a0);
  TMBIR_CHECK_LAUNCH();
  if (int e = conv32(n, n.a0, B, n.wg1, n.master + kOffB1, nullptr, n.a1, true)) return e;
  if (int e = conv32(n, n.a1, B, n.wg2, n.master + kOffB2, nullptr, n.a2, true)) return e;
  k_conv_last<<<blocks, 256, 0, n.stream>>>(n.a2, B, n.H, n.W, n.master, n.out);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

// gradients of sum(gout * net(xin)) added into n.grad; gin (optional, FP32) receives d/dxin
static int net_backward(CnnNet& n, int B, float* gin) {
  const size_t P = (size_t)B * n.H * n.W;
  const int blocks = (int)std::min<size_t>((P + 255) / 256, 152 * 16);
  const int rb = (kW1 + 255) / 256;
  // layer 3
  k_wgrad_last<<<kWgradBlocks, 64, 0, n.stream>>>(n.gout, n.a2, B, n.H, n.W, n.wpart);
  TMBIR_CHECK_LAUNCH();
  k_reduce_parts<<<2, 256, 0, n.stream>>>(n.wpart, kWgradBlocks, kW3 + kB3, n.grad + kOff3);
  TMBIR_CHECK_LAUNCH();
  k_last_dgrad<<<blocks, 256, 0, n.stream>>>(n.gout, n.a2, B, n.H, n.W, n.master, n.g2);
  TMBIR_CHECK_LAUNCH();
  // layer 2: weights from (g2, a1), then g1 = mask(a1) conv(g2, W2 flipped transposed)
  k_wgrad32<<<kWgradBlocks, 256, 0, n.stream>>>(n.g2, n.a1, B, n.H, n.W, n.wpart);
  TMBIR_CHECK_LAUNCH();
  k_reduce_parts<<<rb, 256, 0, n.stream>>>(n.wpart, kWgradBlocks, kW1, n.grad + kOff2);
  TMBIR_CHECK_LAUNCH();
  k_bias_grad<<<kWgradBlocks, 32, 0, n.stream>>>(n.g2, P, n.wpart);
  TMBIR_CHECK_LAUNCH();
  k_reduce_parts<<<1, 32, 0, n.stream>>>(n.wpart, kWgradBlocks, kB1, n.grad + kOffB2);
  TMBIR_CHECK_LAUNCH();
  if (int e = conv32(n, n.g2, B, n.wt2, nullptr, n.a1, n.g1, false)) return e;
  // layer 1: weights from (g1, a0), then g0 = mask(a0) conv(g1, W1 flipped transposed) into g2's buffer
  k_wgrad32<<<kWgradBlocks, 256, 0, n.stream>>>(n.g1, n.a0, B, n.H, n.W, n.wpart);
  TMBIR_CHECK_LAUNCH();
  k_reduce_parts<<<rb, 256, 0, n.stream>>>(n.wpart, kWgradBlocks, kW1, n.grad + kOff1);
  TMBIR_CHECK_LAUNCH();
  k_bias_grad<<<kWgradBlocks, 32, 0, n.stream>>>(n.g1, P, n.wpart);
  TMBIR_CHECK_LAUNCH();
  k_reduce_parts<<<1, 32, 0, n.stream>>>(n.wpart, kWgradBlocks, kB1, n.grad + kOffB1);
  TMBIR_CHECK_LAUNCH();
  __nv_bfloat16* g0 = n.g2;
  if (int e = conv32(n, n.g1, B, n.wt1, nullptr, n.a0, g0, false)) return e;
  // layer 0
  k_wgrad_first<<<kWgradBlocks, 128, 0, n.stream>>>(g0, n.xin, B, n.H, n.W, n.wpart);
  TMBIR_CHECK_LAUNCH();
  k_reduce_parts<<<2, 256, 0, n.stream>>>(n.wpart, kWgradBlocks, kW0 + kB0, n.grad + kOff0);
  TMBIR_CHECK_LAUNCH();
  if (gin) {
    k_first_dgrad<<<blocks, 256, 0, n.stream>>>(g0, B, n.H, n.W, n.master, gin);
    TMBIR_CHECK_LAUNCH();
  }
  return TMBIR_OK;
}

static int pack(CnnNet& n) {
  k_cnn_pack<<<(kWElems + 255) / 256, 256, 0, n.stream>>>(n.master, n.wg1, n.wg2, n.wt1, n.wt2);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

static int normalise(CnnNet& n, const float* x, int B) {
  const int HW = n.H * n.W;
  const size_t P = (size_t)B * HW;
  k_norm_partial<<<dim3(kNormBlocks, B), 256, 0, n.stream>>>(x, HW, n.dpart);
  TMBIR_CHECK_LAUNCH();
  k_norm_stats<<<B, 32, 0, n.stream>>>(n.dpart, HW, n.sig);
  TMBIR_CHECK_LAUNCH();
  k_scale_in<<<(int)std::min<size_t>((P + 255) / 256, 152 * 16), 256, 0, n.stream>>>(x, HW, P, n.sig, n.xin);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

}  // namespace tmbir

using namespace tmbir;

struct tmbir_cnn {
  CnnNet n;
  size_t offs[20];
};

#define CNN_REQUIRE(cond, code, msg) \
  do {                               \
    if (!(cond)) return set_error(code, msg); \
  } while (0)

static bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" {

int tmbir_cnn_param_count(void) { return kParams; }

int tmbir_cnn_workspace_size(int max_batch, int H, int W, size_t* bytes) {
  CNN_REQUIRE(bytes && max_batch >= 1 && H >= 1 && W >= 1 && (size_t)max_batch * H * W < ((size_t)1 << 31),
              TMBIR_ERR_ARG, "cnn_workspace_size: bad sizes");
  size_t offs[20];
  *bytes = cnn_bytes(max_batch, H, W, offs);
  return TMBIR_OK;
}

int tmbir_cnn_create(tmbir_cnn** out, void* stream, int max_batch, int H, int W, void* d_ws, size_t bytes) {
  CNN_REQUIRE(out && d_ws && ((uintptr_t)d_ws & 255u) == 0, TMBIR_ERR_ARG,
              "cnn_create: NULL argument or workspace not 256-byte aligned");
  size_t need = 0;
  if (int e = tmbir_cnn_workspace_size(max_batch, H, W, &need)) return e;
  CNN_REQUIRE(bytes >= need, TMBIR_ERR_WORKSPACE, "cnn_create: workspace too small");
  tmbir_cnn* c = new tmbir_cnn();
  cnn_bytes(max_batch, H, W, c->offs);
  char* ws = static_cast<char*>(d_ws);
  CnnNet& n = c->n;
  n.stream = (cudaStream_t)stream;
  n.max_batch = max_batch;
  n.H = H;
  n.W = W;
  n.master = reinterpret_cast<float*>(ws + c->offs[0]);
  n.grad = reinterpret_cast<float*>(ws + c->offs[1]);
  n.adam_m = reinterpret_cast<float*>(ws + c->offs[2]);
  n.adam_v = reinterpret_cast<float*>(ws + c->offs[3]);
  n.wg1 = reinterpret_cast<__nv_bfloat16*>(ws + c->offs[4]);
  n.wg2 = reinterpret_cast<__nv_bfloat16*>(ws + c->offs[5]);
  n.wt1 = reinterpret_cast<__nv_bfloat16*>(ws + c->offs[6]);
  n.wt2 = reinterpret_cast<__nv_bfloat16*>(ws + c->offs[7]);
  n.a0 = reinterpret_cast<__nv_bfloat16*>(ws + c->offs[8]);
  n.a1 = reinterpret_cast<__nv_bfloat16*>(ws + c->offs[9]);
  n.a2 = reinterpret_cast<__nv_bfloat16*>(ws + c->offs[10]);
  n.g1 = reinterpret_cast<__nv_bfloat16*>(ws + c->offs[11]);
  n.g2 = reinterpret_cast<__nv_bfloat16*>(ws + c->offs[12]);
  n.xin = reinterpret_cast<float*>(ws + c->offs[13]);
  n.out = reinterpret_cast<float*>(ws + c->offs[14]);
  n.gout = reinterpret_cast<float*>(ws + c->offs[15]);
  n.sig = reinterpret_cast<float*>(ws + c->offs[16]);
  n.wpart = reinterpret_cast<float*>(ws + c->offs[17]);
  n.dpart = reinterpret_cast<double*>(ws + c->offs[18]);
  n.err = reinterpret_cast<int*>(ws + c->offs[19]);
  if (cudaMemsetAsync(n.err, 0, sizeof(int), n.stream) != cudaSuccess) {
    delete c;
    return set_error(TMBIR_ERR_CUDA, "cnn_create: cudaMemsetAsync failed");
  }
  n.step = 0;
  *out = c;
  return TMBIR_OK;
}

int tmbir_cnn_destroy(tmbir_cnn* net) {
  delete net;
  return TMBIR_OK;
}

int tmbir_cnn_set_weights(tmbir_cnn* net, const float* h_params) {
  CNN_REQUIRE(net && h_params, TMBIR_ERR_ARG, "cnn_set_weights: NULL argument");
  CnnNet& n = net->n;
  TMBIR_CUDA(cudaMemcpyAsync(n.master, h_params, kParams * sizeof(float), cudaMemcpyHostToDevice, n.stream));
  TMBIR_CUDA(cudaMemsetAsync(n.adam_m, 0, kParams * sizeof(float), n.stream));
  TMBIR_CUDA(cudaMemsetAsync(n.adam_v, 0, kParams * sizeof(float), n.stream));
  n.step = 0;
  if (int e = pack(n)) return e;
  TMBIR_CUDA(cudaStreamSynchronize(n.stream));
  return TMBIR_OK;
}

int tmbir_cnn_get_weights(tmbir_cnn* net, float* h_params) {
  CNN_REQUIRE(net && h_params, TMBIR_ERR_ARG, "cnn_get_weights: NULL argument");
  CnnNet& n = net->n;
  TMBIR_CUDA(cudaMemcpyAsync(h_params, n.master, kParams * sizeof(float), cudaMemcpyDeviceToHost, n.stream));
  TMBIR_CUDA(cudaStreamSynchronize(n.stream));
  return TMBIR_OK;
}

int tmbir_cnn_init(tmbir_cnn* net, unsigned long long seed) {
  CNN_REQUIRE(net, TMBIR_ERR_ARG, "cnn_init: NULL argument");
  std::mt19937_64 rng(seed);
  std::vector<float> p(kParams, 0.f);
  auto fill = [&](int off, int count, int fan_in, float gain) {
    std::normal_distribution<double> nd(0.0, gain * std::sqrt(2.0 / fan_in));
    for (int i = 0; i < count; ++i) p[off + i] = (float)nd(rng);
  };
  fill(kOff0, kW0, 9, 1.f);
  fill(kOff1, kW1, 9 * kC, 1.f);
  fill(kOff2, kW1, 9 * kC, 1.f);
  fill(kOff3, kW3, 9 * kC, 0.1f);  // small last layer: the refiner starts close to the identity
  return tmbir_cnn_set_weights(net, p.data());
}

int tmbir_cnn_net_forward(tmbir_cnn* net, const float* d_in, int batch, float* d_out) {
  TMBIR_TRACE("tmbir_cnn_net_forward");
  CNN_REQUIRE(net && d_in && d_out && al16(d_in) && al16(d_out), TMBIR_ERR_ARG, "cnn_net_forward: bad buffers");
  CnnNet& n = net->n;
  CNN_REQUIRE(batch >= 1 && batch <= n.max_batch, TMBIR_ERR_ARG, "cnn_net_forward: batch out of range");
  const size_t P = (size_t)batch * n.H * n.W;
  TMBIR_CUDA(cudaMemcpyAsync(n.xin, d_in, P * sizeof(float), cudaMemcpyDeviceToDevice, n.stream));
  if (int e = net_forward(n, batch)) return e;
  TMBIR_CUDA(cudaMemcpyAsync(d_out, n.out, P * sizeof(float), cudaMemcpyDeviceToDevice, n.stream));
  return TMBIR_OK;
}

int tmbir_cnn_net_backward(tmbir_cnn* net, const float* d_in, const float* d_gout, int batch, float* h_gparams,
                           float* d_gin) {
  TMBIR_TRACE("tmbir_cnn_net_backward");
  CNN_REQUIRE(net && d_in && d_gout && h_gparams && al16(d_in) && al16(d_gout) && (!d_gin || al16(d_gin)),
              TMBIR_ERR_ARG, "cnn_net_backward: bad buffers");
  CnnNet& n = net->n;
  CNN_REQUIRE(batch >= 1 && batch <= n.max_batch, TMBIR_ERR_ARG, "cnn_net_backward: batch out of range");
  const size_t P = (size_t)batch * n.H * n.W;
  TMBIR_CUDA(cudaMemcpyAsync(n.xin, d_in, P * sizeof(float), cudaMemcpyDeviceToDevice, n.stream));
  if (int e = net_forward(n, batch)) return e;
  TMBIR_CUDA(cudaMemcpyAsync(n.gout, d_gout, P * sizeof(float), cudaMemcpyDeviceToDevice, n.stream));
  TMBIR_CUDA(cudaMemsetAsync(n.grad, 0, kParams * sizeof(float), n.stream));
  if (int e = net_backward(n, batch, d_gin)) return e;
  TMBIR_CUDA(cudaMemcpyAsync(h_gparams, n.grad, kParams * sizeof(float), cudaMemcpyDeviceToHost, n.stream));
  return check_tc(n);
}

int tmbir_cnn_apply(tmbir_cnn* net, const float* d_x, int batch, float* d_y) {
  TMBIR_TRACE("tmbir_cnn_apply");
  CNN_REQUIRE(net && d_x && d_y && al16(d_x) && al16(d_y), TMBIR_ERR_ARG, "cnn_apply: bad buffers");
  CnnNet& n = net->n;
  CNN_REQUIRE(batch >= 1 && batch <= n.max_batch, TMBIR_ERR_ARG, "cnn_apply: batch out of range");
  const size_t P = (size_t)batch * n.H * n.W;
  if (int e = normalise(n, d_x, batch)) return e;
  if (int e = net_forward(n, batch)) return e;
  k_residual_out<<<(int)std::min<size_t>((P + 255) / 256, 152 * 16), 256, 0, n.stream>>>(d_x, n.out, n.H * n.W, P,
                                                                                        n.sig, d_y);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

int tmbir_cnn_train_step(tmbir_cnn* net, const float* d_x, const float* d_target, int batch, float lr, double* h_loss) {
  TMBIR_TRACE("tmbir_cnn_train_step");
  CNN_REQUIRE(net && d_x && d_target && al16(d_x) && al16(d_target), TMBIR_ERR_ARG, "cnn_train_step: bad buffers");
  CnnNet& n = net->n;
  CNN_REQUIRE(batch >= 1 && batch <= n.max_batch && lr > 0.f, TMBIR_ERR_ARG, "cnn_train_step: bad batch or rate");
  const size_t P = (size_t)batch * n.H * n.W;
  if (int e = normalise(n, d_x, batch)) return e;
  if (int e = net_forward(n, batch)) return e;
  const int lb = 1024;
  k_loss<<<lb, 256, 0, n.stream>>>(n.out, d_x, d_target, n.H * n.W, P, n.sig, n.gout, n.dpart);
  TMBIR_CHECK_LAUNCH();
  k_sum_d<<<1, 32, 0, n.stream>>>(n.dpart, lb, 1.0 / (double)P, n.dpart + lb);
  TMBIR_CHECK_LAUNCH();
  TMBIR_CUDA(cudaMemsetAsync(n.grad, 0, kParams * sizeof(float), n.stream));
  if (int e = net_backward(n, batch, nullptr)) return e;
  n.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n.step), c2 = 1.f - std::pow(b2, (float)n.step);
  k_adam<<<(kParams + 255) / 256, 256, 0, n.stream>>>(n.master, n.grad, n.adam_m, n.adam_v, kParams, lr, b1, b2, 1e-8f,
                                                      c1, c2);
  TMBIR_CHECK_LAUNCH();
  if (int e = pack(n)) return e;
  if (h_loss) {
    TMBIR_CUDA(cudaMemcpyAsync(h_loss, n.dpart + lb, sizeof(double), cudaMemcpyDeviceToHost, n.stream));
    return check_tc(n);
  }
  return TMBIR_OK;
}

int tmbir_warm_start(tmbir_ctx* ctx, tmbir_cnn* net, const float* d_fbp, const float* d_atg, const tmbir_params* prm,
                     float* d_x0, int* h_used_cnn) {
  TMBIR_TRACE("tmbir_warm_start");
  CNN_REQUIRE(ctx && net && d_fbp && d_atg && prm && d_x0 && al16(d_fbp) && al16(d_x0), TMBIR_ERR_ARG,
              "warm_start: bad arguments");
  CNN_REQUIRE(d_x0 != d_fbp, TMBIR_ERR_ARG, "warm_start: output must not alias the FBP start");
  Ctx& c = ctx->c;
  CnnNet& n = net->n;
  CNN_REQUIRE(c.groups.size() == 1 && c.groups[0].N == n.H && n.H == n.W, TMBIR_ERR_SHAPE,
              "warm_start: needs one geometry group whose N equals the network's image size");
  const int S = c.groups[0].n_slices;
  const size_t HW = (size_t)n.H * n.W;
  // the network runs on its own stream: it starts after the context's pending work and the
  // objectives below start after it
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (n.stream != c.stream) {
    TMBIR_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    if (cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaEventDestroy(ev[0]);
      return set_error(TMBIR_ERR_CUDA, "warm_start: cudaEventCreate failed");
    }
  }
  auto release = [&](int e) {
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    return e;
  };
  if (ev[0]) {
    if (cudaEventRecord(ev[0], c.stream) != cudaSuccess || cudaStreamWaitEvent(n.stream, ev[0], 0) != cudaSuccess)
      return release(set_error(TMBIR_ERR_CUDA, "warm_start: stream ordering failed"));
  }
  for (int s0 = 0; s0 < S; s0 += n.max_batch) {
    const int b = std::min(n.max_batch, S - s0);
    if (int e = tmbir_cnn_apply(net, d_fbp + s0 * HW, b, d_x0 + s0 * HW)) return release(e);
  }
  if (ev[1]) {
    if (cudaEventRecord(ev[1], n.stream) != cudaSuccess || cudaStreamWaitEvent(c.stream, ev[1], 0) != cudaSuccess)
      return release(set_error(TMBIR_ERR_CUDA, "warm_start: stream ordering failed"));
  }
  release(0);
  double F_cnn = 0.0, F_fbp = 0.0;
  if (int e = tmbir_objective(ctx, d_x0, d_atg, prm, &F_cnn)) return e;
  if (int e = tmbir_objective(ctx, d_fbp, d_atg, prm, &F_fbp)) return e;
  const int use = F_cnn < F_fbp ? 1 : 0;
  if (!use) TMBIR_CUDA(cudaMemcpyAsync(d_x0, d_fbp, S * HW * sizeof(float), cudaMemcpyDeviceToDevice, c.stream));
  if (h_used_cnn) *h_used_cnn = use;
  return check_tc(n);
}

}  // extern "C"
