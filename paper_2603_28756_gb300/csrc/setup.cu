// Setup of the Toeplitz operator (Sec. 2.1) and the back-projection used for R*g and the
// FBP start (Sec. 2.2), both through a type-1 non-uniform FFT (Eq. 4).
//
// Polar samples xi_{a,k} = (k / n_det) (cos theta_a, sin theta_a), |k| <= n_det/2 - 1.
//   K(d)    = (1/n_det) sum_{a,k} exp(+2 pi i xi . d),               d in [-(N-1), N-1]^2
//   R*g(x)  = (1/n_det) sum_{a,k} G(a,k) exp(-2 pi i xi . x),       G(a,k) = sum_m g(a,m) exp(2 pi i k s_m / n_det)
// The type-1 transform spreads the samples onto an oversampled periodic grid with the
// "exponential of semicircle" kernel psi(u) = exp(beta (sqrt(1 - (2u/w)^2) - 1)) (Barnett,
// Magland & af Klinteberg 2019), takes a 2D FFT and divides each output mode by the
// kernel's Fourier transform.  K (4N grid, width 12) and R*g (5N/4 grid, width 14) run in
// FP64, the FBP start (2N grid, width 10) in FP32.  K is spread with fixed-point integer atomics and R*g / FBP through a sorted sparse
// matrix, so every result is bit-reproducible.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fft.cuh"
#include "internal.h"

namespace tmbir {

// ---------------------------------------------------------------- batched 1D FFT along rows
// Stockham autosort in shared memory: one block per row, radix 8/4/2/3/5 stages, natural order
// in and out.  tw[j] = exp(-2 pi i j / n).
template <int R, int DIR, class C>
__device__ __forceinline__ void stockham_stage(const C* X, C* Y, int n, int Ls, const C* __restrict__ tw) {
  const int nb = n / R;
  const int tstep = n / (Ls * R);
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int k = j % Ls;  // Ls is a product of mixed radices
    C a[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      C v = X[j + m * nb];
      if (m > 0 && k > 0) {
        const C w = tw[(size_t)k * m * tstep];  // k m tstep < n
        v = DIR < 0 ? cmul(v, w) : cmulc(v, w);
      }
      a[m] = v;
    }
    reg_dft<R, DIR, C>(a);
    const int o = (j - k) * R + k;
#pragma unroll
    for (int m = 0; m < R; ++m) Y[o + m * Ls] = a[m];
  }
}

// X[perm(j)] = row[j] for j < n, in batches of eight loads per thread issued before their stores
// (a long row fills a block alone, so nothing else on the SM hides the load latency)
template <class C, class Perm>
__device__ __forceinline__ void load_row(const C* __restrict__ row, C* X, int n, Perm perm) {
  for (int j0 = threadIdx.x; j0 < n; j0 += 8 * blockDim.x) {
    C v[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int j = j0 + b * blockDim.x;
      if (j < n) v[b] = row[j];
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int j = j0 + b * blockDim.x;
      if (j < n) X[perm(j)] = v[b];
    }
  }
}

// plan: the radices, one per 4-bit digit from the lowest (built by fft_plan)
template <int DIR, class C>
__global__ void __launch_bounds__(256) k_fft_rows(C* data, int n, unsigned plan, size_t stride, const C* __restrict__ tw) {
  extern __shared__ unsigned char smraw[];
  C* X = reinterpret_cast<C*>(smraw);
  C* Y = X + n;
  C* row = data + (size_t)blockIdx.x * stride;
  load_row(row, X, n, [](int j) { return j; });
  __syncthreads();
  int Ls = 1;
  for (; plan != 0; plan >>= 4) {
    const int R = (int)(plan & 15u);
    switch (R) {
      case 8: stockham_stage<8, DIR>(X, Y, n, Ls, tw); break;
      case 4: stockham_stage<4, DIR>(X, Y, n, Ls, tw); break;
      case 2: stockham_stage<2, DIR>(X, Y, n, Ls, tw); break;
      case 3: stockham_stage<3, DIR>(X, Y, n, Ls, tw); break;
      default: stockham_stage<5, DIR>(X, Y, n, Ls, tw); break;
    }
    Ls *= R;
    __syncthreads();
    C* tmp = X;
    X = Y;
    Y = tmp;
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] = X[j];
}

// In-place variant for rows whose two Stockham buffers do not fit in shared memory: the row
// is loaded in bit-reversed order, then log2(n) radix-2 decimation-in-time stages.
template <int DIR, class C>
__global__ void __launch_bounds__(1024) k_fft_rows_inplace(C* data, int n, int log2n, size_t stride,
                                                           const C* __restrict__ tw) {
  extern __shared__ unsigned char smraw[];
  C* X = reinterpret_cast<C*>(smraw);
  C* row = data + (size_t)blockIdx.x * stride;
  load_row(row, X, n, [log2n](int j) { return (int)(__brev((unsigned)j) >> (32 - log2n)); });
  __syncthreads();
  for (int half = 1, tstep = n / 2; half < n; half <<= 1, tstep >>= 1) {
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const int k = b & (half - 1);
      const int i0 = 2 * (b - k) + k, i1 = i0 + half;
      const C w = tw[(size_t)k * tstep];
      const C v = DIR < 0 ? cmul(X[i1], w) : cmulc(X[i1], w);
      const C u = X[i0];
      X[i0] = cadd(u, v);
      X[i1] = csub(u, v);
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] = X[j];
}

// out[b][c][r] = in[b][r][c] for a batch of rows x cols matrices
template <class C>
__global__ void k_transpose(const C* __restrict__ in, C* __restrict__ out, int rows, int cols) {
  __shared__ C tile[32][33];
  const size_t boff = (size_t)blockIdx.z * rows * cols;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = in[boff + (size_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[boff + (size_t)c * rows + r] = tile[threadIdx.x][i];
  }
}

static int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}
// radices of n = 2^a 3^b 5^c as 4-bit digits (fives and threes first, then eights, fours,
// twos); 0 when n has another factor or needs more than eight stages
static unsigned fft_plan(int n) {
  unsigned plan = 0;
  int shift = 0;
  auto push = [&](int r) {
    plan |= (unsigned)r << shift;
    shift += 4;
  };
  while (n % 5 == 0) { push(5); n /= 5; }
  while (n % 3 == 0) { push(3); n /= 3; }
  while (n % 8 == 0) { push(8); n /= 8; }
  if (n % 4 == 0) { push(4); n /= 4; }
  if (n % 2 == 0) { push(2); n /= 2; }
  return (n == 1 && shift <= 32) ? plan : 0u;
}

template <class C>
static int fft_rows(C* data, int n, int rows, int dir, const C* tw, cudaStream_t s) {
  const size_t smem = 2 * (size_t)n * sizeof(C);
  static bool attr_set = false;
  if (!attr_set) {
    TMBIR_CUDA(cudaFuncSetAttribute(k_fft_rows<-1, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    TMBIR_CUDA(cudaFuncSetAttribute(k_fft_rows<1, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    TMBIR_CUDA(cudaFuncSetAttribute(k_fft_rows_inplace<-1, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024));
    TMBIR_CUDA(cudaFuncSetAttribute(k_fft_rows_inplace<1, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024));
    attr_set = true;
  }
  if (smem > 200 * 1024) {
    if (smem / 2 > 200 * 1024 || (n & (n - 1)) != 0) return set_error(TMBIR_ERR_SHAPE, "setup FFT length too large");
    if (dir < 0)
      k_fft_rows_inplace<-1, C><<<rows, 1024, smem / 2, s>>>(data, n, ilog2(n), (size_t)n, tw);
    else
      k_fft_rows_inplace<1, C><<<rows, 1024, smem / 2, s>>>(data, n, ilog2(n), (size_t)n, tw);
    TMBIR_CHECK_LAUNCH();
    return TMBIR_OK;
  }
  const unsigned plan = fft_plan(n);
  if (!plan) return set_error(TMBIR_ERR_SHAPE, "setup FFT length must be 2^a 3^b 5^c");
  if (dir < 0)
    k_fft_rows<-1, C><<<rows, 256, smem, s>>>(data, n, plan, (size_t)n, tw);
  else
    k_fft_rows<1, C><<<rows, 256, smem, s>>>(data, n, plan, (size_t)n, tw);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

template <class C>
static int transpose(const C* in, C* out, int rows, int cols, int batch, cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch), block(32, 8);
  k_transpose<C><<<grid, block, 0, s>>>(in, out, rows, cols);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

// 2D FFT of `batch` n x n grids; result left transposed in `tmp` (tmp[b][kx][ky]).
template <class C>
static int fft2_transposed(C* grid, C* tmp, int n, int batch, int dir, const C* tw, cudaStream_t s) {
  if (int e = fft_rows(grid, n, n * batch, dir, tw, s)) return e;
  if (int e = transpose(grid, tmp, n, n, batch, s)) return e;
  return fft_rows(tmp, n, n * batch, dir, tw, s);
}

// ---------------------------------------------------------------- spreading
__device__ __forceinline__ double es_kernel(double z, double beta) {  // z in [-1, 1]
  const double t = 1.0 - z * z;
  return t > 0.0 ? exp(beta * (sqrt(t) - 1.0)) : 0.0;
}
// Spreading of the constant strength 1/n_det (the kernel K) with 64-bit fixed-point integer
// atomics: integer addition is associative, so the grid is bit-identical run to run.  Every
// cell sum is below 2 (at most ~2 n_det points of weight <= 1/n_det each reach one cell), so a
// scale of 2^52 keeps ~1e-16 absolute resolution without overflow.
constexpr double kFixScale = 4503599627370496.0;  // 2^52
template <int W>
__global__ void k_spread_fixed(const double* __restrict__ angles, int na, int nd, int nf,
                               unsigned long long* __restrict__ grid, double beta, const double* __restrict__ wts) {
  const int npa = nd - 1;
  const size_t total = (size_t)na * npa;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const int kk = (int)(id % npa), a = (int)(id / npa);
    const int k = kk - (nd / 2 - 1);
    double sa, ca;
    sincos(angles[a], &sa, &ca);
    const double ux = (double)k * ca * nf / nd, uy = (double)k * sa * nf / nd;
    const int lx0 = (int)ceil(ux - 0.5 * W), ly0 = (int)ceil(uy - 0.5 * W);
    double kx[W], ky[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
      kx[j] = es_kernel((2.0 * (lx0 + j - ux)) / W, beta);
      ky[j] = es_kernel((2.0 * (ly0 + j - uy)) / W, beta);
    }
    const double c = kFixScale / nd * (wts ? wts[a] : 1.0);  // weights in [0, 1] keep the bound
#pragma unroll 1
    for (int jy = 0; jy < W; ++jy) {
      const int ly = (ly0 + jy + nf) % nf;
#pragma unroll
      for (int jx = 0; jx < W; ++jx) {
        const int lx = (lx0 + jx + nf) % nf;
        atomicAdd(&grid[(size_t)ly * nf + lx], (unsigned long long)(long long)llrint(c * ky[jy] * kx[jx]));
      }
    }
  }
}
__global__ void k_fixed_to_complex(const unsigned long long* __restrict__ in, double2* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_double2((double)(long long)in[i] / kFixScale, 0.0);
}

// ---------------------------------------------------------------- sparse spreading operator
// The polar sample positions depend on the geometry only, so the spreading onto the 2N x 2N
// grid of R*g and of the FBP start is stored once as a sparse matrix in compressed rows, one
// row per grid cell: the strength index a * n_det + (k mod n_det) of every contributing
// sample and its kernel weight psi(x) psi(y).  Entries of a row are sorted by strength index,
// so every later gather sums in a fixed order (deterministic) and needs no atomics.
__global__ void k_csr_count(const double* __restrict__ angles, int na, int nd, int nf, int W, int* __restrict__ cnt) {
  const int npa = nd - 1;
  const size_t total = (size_t)na * npa;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const int kk = (int)(id % npa), a = (int)(id / npa);
    const int k = kk - (nd / 2 - 1);
    double sa, ca;
    sincos(angles[a], &sa, &ca);
    const double ux = (double)k * ca * nf / nd, uy = (double)k * sa * nf / nd;
    const int lx0 = (int)ceil(ux - 0.5 * W), ly0 = (int)ceil(uy - 0.5 * W);
    for (int jy = 0; jy < W; ++jy)
      for (int jx = 0; jx < W; ++jx) {
        const int ly = (ly0 + jy + nf) % nf, lx = (lx0 + jx + nf) % nf;
        atomicAdd(&cnt[(size_t)ly * nf + lx + 1], 1);
      }
  }
}
__global__ void k_csr_fill(const double* __restrict__ angles, int na, int nd, int nf, int W, double beta,
                           int* __restrict__ cursor, int* __restrict__ idx, double* __restrict__ wt) {
  const int npa = nd - 1;
  const size_t total = (size_t)na * npa;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const int kk = (int)(id % npa), a = (int)(id / npa);
    const int k = kk - (nd / 2 - 1);
    double sa, ca;
    sincos(angles[a], &sa, &ca);
    const double ux = (double)k * ca * nf / nd, uy = (double)k * sa * nf / nd;
    const int lx0 = (int)ceil(ux - 0.5 * W), ly0 = (int)ceil(uy - 0.5 * W);
    const int sidx = a * nd + (k < 0 ? k + nd : k);
    for (int jy = 0; jy < W; ++jy) {
      const double wy = es_kernel((2.0 * (ly0 + jy - uy)) / W, beta);
      for (int jx = 0; jx < W; ++jx) {
        const int ly = (ly0 + jy + nf) % nf, lx = (lx0 + jx + nf) % nf;
        const int pos = atomicAdd(&cursor[(size_t)ly * nf + lx], 1);
        idx[pos] = sidx;
        wt[pos] = wy * es_kernel((2.0 * (lx0 + jx - ux)) / W, beta);
      }
    }
  }
}
// insertion sort of each row by strength index (rows are short except near the centre)
__global__ void k_csr_sort(const int* __restrict__ ptr, int ncells, int* __restrict__ idx, double* __restrict__ wt) {
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < ncells; cell += gridDim.x * blockDim.x) {
    const int b = ptr[cell], e = ptr[cell + 1];
    for (int i = b + 1; i < e; ++i) {
      const int ki = idx[i];
      const double wi = wt[i];
      int j = i - 1;
      while (j >= b && idx[j] > ki) {
        idx[j + 1] = idx[j];
        wt[j + 1] = wt[j];
        --j;
      }
      idx[j + 1] = ki;
      wt[j + 1] = wi;
    }
  }
}
// inclusive scan, three phases over tiles of 2048 ints
__global__ void k_scan_tiles(int* __restrict__ a, int n, int* __restrict__ sums) {
  __shared__ int sh[2048];
  const int base = blockIdx.x * 2048;
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) sh[i] = base + i < n ? a[base + i] : 0;
  __syncthreads();
  for (int off = 1; off < 2048; off <<= 1) {
    int v[8];
    for (int r = 0; r < 8; ++r) {
      const int i = threadIdx.x + r * 256;
      v[r] = i >= off ? sh[i - off] : 0;
    }
    __syncthreads();
    for (int r = 0; r < 8; ++r) sh[threadIdx.x + r * 256] += v[r];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < 2048; i += blockDim.x)
    if (base + i < n) a[base + i] = sh[i];
  if (threadIdx.x == 0) sums[blockIdx.x] = sh[2047];
}
__global__ void k_scan_sums(int* sums, int nt) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    for (int i = 1; i < nt; ++i) sums[i] += sums[i - 1];
}
__global__ void k_scan_add(int* __restrict__ a, int n, const int* __restrict__ sums) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int t = i / 2048;
    if (t > 0) a[i] += sums[t - 1];
  }
}
// a weight of the sparse spreading matrix as the arithmetic's real type: FP64 and FP32 read the
// double; the double-word matrix holds each weight as an (hi, lo) pair of floats in its 8 bytes
template <class S>
__device__ __forceinline__ S load_wt(const double* wt, int j) {
  return (S)wt[j];
}
template <>
__device__ __forceinline__ df load_wt<df>(const double* wt, int j) {
  const float2 w = __ldg(reinterpret_cast<const float2*>(wt) + j);
  return df(w.x, w.y);
}
// in place: every double weight of a spreading matrix becomes its double-word (hi, lo)
__global__ void k_wt_to_df(double* wt, size_t n) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    const df w(wt[j]);
    reinterpret_cast<float2*>(wt)[j] = make_float2(w.hi, w.lo);
  }
}

// grid[b][cell] = sum_j wt[j] strengths[idx[j]][b], B slices per launch (sample-major strengths)
template <int B, class C>
__global__ void k_csr_gather(const int* __restrict__ ptr, const int* __restrict__ idx, const double* __restrict__ wt,
                             int ncells, const C* __restrict__ strengths, C* __restrict__ grid, int nb) {
  using S = real_t<C>;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < ncells; cell += gridDim.x * blockDim.x) {
    C acc[B];
#pragma unroll
    for (int b = 0; b < B; ++b) acc[b] = mkc((S)0, (S)0);
    const int e = ptr[cell + 1];
    int j = ptr[cell];
    // two entries per step with all their loads issued first (the index load and the dependent
    // strength loads are a latency chain); the accumulation order is that of one at a time
    for (; j + 1 < e; j += 2) {
      const C* sv0 = strengths + (size_t)idx[j] * B;
      const C* sv1 = strengths + (size_t)idx[j + 1] * B;
      const S w0 = load_wt<S>(wt, j), w1 = load_wt<S>(wt, j + 1);
      C v0[B], v1[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        v0[b] = sv0[b];
        v1[b] = sv1[b];
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        acc[b].x = fmar(w0, v0[b].x, acc[b].x);
        acc[b].y = fmar(w0, v0[b].y, acc[b].y);
        acc[b].x = fmar(w1, v1[b].x, acc[b].x);
        acc[b].y = fmar(w1, v1[b].y, acc[b].y);
      }
    }
    if (j < e) {
      const C* sv = strengths + (size_t)idx[j] * B;
      const S w = load_wt<S>(wt, j);
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const C v = sv[b];
        acc[b].x = fmar(w, v.x, acc[b].x);
        acc[b].y = fmar(w, v.y, acc[b].y);
      }
    }
#pragma unroll
    for (int b = 0; b < B; ++b)
      if (b < nb) grid[(size_t)b * ncells + cell] = acc[b];
  }
}
// tmp[b][j][r] = grid[b][r][(j - N/2) mod nf] for the N kept x-modes j (column pruning)
template <class C>
__global__ void k_transpose_prune(const C* __restrict__ in, C* __restrict__ out, int nf, int N) {
  __shared__ C tile[32][33];
  const size_t ib = (size_t)blockIdx.z * nf * nf, ob = (size_t)blockIdx.z * N * nf;
  const int j0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, j = j0 + threadIdx.x;
    if (r < nf && j < N) tile[i][threadIdx.x] = in[ib + (size_t)r * nf + ((j - N / 2 + nf) % nf)];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int j = j0 + i, r = r0 + threadIdx.x;
    if (r < nf && j < N) out[ob + (size_t)j * nf + r] = tile[threadIdx.x][i];
  }
}
// out[b][r][c] = scale * Re tmp[b][c][(r - N/2) mod nf] / (psi[c] psi[r])
// slice 2p from the real part, slice 2p + 1 (when there is one) from the imaginary part of pair p.
// tmp is column-major ([c][r']) and out row-major, so 32 x 32 tiles pass through shared memory
// and both sides are read and written along their contiguous index.  Grid: (N/32, N/32, pairs).
template <class C>
__global__ void __launch_bounds__(256) k_deconv_pruned(const C* __restrict__ B, int nf, int N, int nb,
                                                       const double* __restrict__ psi, float scale,
                                                       float* __restrict__ out) {
  __shared__ C tile[32][33];
  __shared__ double inv_r[32], inv_c[32];  // 1 / psi of the tile's rows and columns
  const int p = blockIdx.z, c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const C* Bp = B + (size_t)p * N * nf;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {  // column c0 + i, rows r0 .. r0 + 31
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < N && r < N) tile[i][threadIdx.x] = Bp[(size_t)c * nf + (r - N / 2 + nf) % nf];
  }
  if (threadIdx.y == 0) {  // one division per row and column of the tile instead of one per pixel
    const int r = r0 + threadIdx.x, c = c0 + threadIdx.x;
    inv_r[threadIdx.x] = r < N ? 1.0 / psi[r] : 0.0;
    inv_c[threadIdx.x] = c < N ? 1.0 / psi[c] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {  // row r0 + i, columns c0 .. c0 + 31
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (c >= N || r >= N) continue;
    const C v = tile[threadIdx.x][i];
    const double f = scale * inv_c[threadIdx.x] * inv_r[i];
    out[((size_t)(2 * p) * N + r) * N + c] = (float)((double)v.x * f);
    if (2 * p + 1 < nb) out[((size_t)(2 * p + 1) * N + r) * N + c] = (float)((double)v.y * f);
  }
}

// K[(dy+N-1)(2N-1) + dx+N-1] = Re B[dx][dy] / (psi(dx) psi(dy)); B transposed ([kx][ky]).
__global__ void k_deconv_K(const double2* __restrict__ B, int nf, int N, const double* __restrict__ psi, double* K) {
  const int W = 2 * N - 1;
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < W * W; id += gridDim.x * blockDim.x) {
    const int ix = id % W, iy = id / W;
    const int dx = ix - (N - 1), dy = iy - (N - 1);
    const double2 v = B[(size_t)((dx + nf) % nf) * nf + (dy + nf) % nf];
    K[id] = v.x / (psi[ix] * psi[iy]);
  }
}

// circulant embedding of K in an M x M grid (M = 2N), complex FP64, [row = y][col = x]
__global__ void k_circulant(const double* __restrict__ K, int N, double2* Cg) {
  const int M = 2 * N, W = 2 * N - 1;
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < M * M; id += gridDim.x * blockDim.x) {
    const int x = id % M, y = id / M;
    const int dx = x < N ? x : x - M, dy = y < N ? y : y - M;  // x == N (d = +-N) is never read by the crop
    double v = 0.0;
    if (dx > -N && dx < N && dy > -N && dy < N) v = K[(dy + N - 1) * W + dx + N - 1];
    Cg[id] = make_double2(v, 0.0);
  }
}

// chat[v][h][k] = Re C_hat[u = 2k + h][v] / M^2, spectrum transposed ([kx = v][ky = u])
__global__ void k_chat_layout(const double2* __restrict__ B, int N, float* chat) {
  const int M = 2 * N;
  const size_t total = (size_t)(N + 1) * 2 * N;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(id % N), h = (int)((id / N) % 2), v = (int)(id / (2 * (size_t)N));
    const int u = 2 * k + h;
    chat[id] = (float)(B[(size_t)v * M + u].x / ((double)M * (double)M));
  }
}

// real sinogram rows -> complex rows for the radial FFT, optional ramp filter (Eq. 12 with the
// unit-pitch Ram-Lak kernel h[0] = 1/4, h[odd n] = -1/(pi^2 n^2), h[even n != 0] = 0; linear
// convolution over the detector, FP32 -- only the FBP start uses it)
template <class C>
__global__ void k_prepare_rows(const float* __restrict__ sino, int nd, size_t rows, int ramp, C* out) {
  extern __shared__ float srow[];
  float* htab = srow + nd;
  using S = real_t<C>;
  if (ramp) {
    for (int n = threadIdx.x; n < nd; n += blockDim.x)
      htab[n] = (n & 1) ? (float)(-1.0 / (M_PI * M_PI * (double)n * (double)n)) : 0.f;
  }
  for (size_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const float* g = sino + row * nd;
    __syncthreads();
    for (int m = threadIdx.x; m < nd; m += blockDim.x) srow[m] = g[m];
    __syncthreads();
    for (int m = threadIdx.x; m < nd; m += blockDim.x) {
      float v = srow[m];
      if (ramp) {
        float acc = 0.25f * srow[m];
        for (int m2 = (m & 1) ? 0 : 1; m2 < nd; m2 += 2) acc = fmaf(srow[m2], htab[m > m2 ? m - m2 : m2 - m], acc);
        v = acc;
      }
      out[row * nd + m] = mkc((S)v, (S)0);
    }
  }
}

// G(a,k) = (-1)^k * sum_m g(a,m) exp(+2 pi i k m / nd) / nd: sign flip from s_m = m - nd/2, and the 1/nd of R*.
// Two slices share one transform: G_pair = G_{2p} + i G_{2p+1}.  Each slice's strengths are
// Hermitian in k (real sinogram, samples symmetric in k), so its gridded transform is real and
// the pair's result carries slice 2p in the real and slice 2p+1 in the imaginary part.
// Written sample-major, out[(a nd + k) PB + p], so the gather reads the PB pairs of a sample
// from one contiguous run.
// wts: per-angle weights of the data term (R* W g; nullptr: none), angle = r / nd.
template <int PB, class C>
__global__ void k_strength_pack(const C* __restrict__ rows, int nd, size_t nrows, int nb, C* __restrict__ out,
                                const double* __restrict__ wts) {
  using S = real_t<C>;
  const size_t total = nrows * PB;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const int pr = (int)(id % PB);
    const size_t r = id / PB;
    const int k = (int)(r % nd);
    const double w = wts ? wts[r / nd] / nd : 1.0 / nd;
    const S sg = (k & 1) ? (S)(-w) : (S)w;
    const C a = 2 * pr < nb ? rows[(size_t)(2 * pr) * nrows + r] : mkc((S)0, (S)0);
    const C b = 2 * pr + 1 < nb ? rows[(size_t)(2 * pr + 1) * nrows + r] : mkc((S)0, (S)0);
    out[id] = mkc((a.x - b.y) * sg, (a.y + b.x) * sg);
  }
}

// 1/2 sum x^2: each block reduces a strided share in FP64 (fixed order), then one block sums
// the block partials in order.
__global__ void k_sumsq_blocks(const float* __restrict__ x, size_t n, double* part, const double* __restrict__ wts,
                               int na, int nd) {
  __shared__ double sh[256];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    s += wts ? wts[(i / nd) % na] * (v * v) : v * v;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void k_sum_half(const double* __restrict__ part, int n, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 0.5 * sh[0];
}

// ---------------------------------------------------------------- power iteration helpers
__global__ void k_fill(float* x, size_t n, float v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] = v;
}
// v = w / ||w||, ||w||^2 = sums[5];  lam = sums[0] (v.w)
__global__ void k_normalize(const float* __restrict__ w, float* __restrict__ v, size_t n, const double* sums, double* lam) {
  const double nrm = sqrt(sums[5]);
  const float inv = (float)(1.0 / nrm);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) v[i] = w[i] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) *lam = sums[0];
}

// ---------------------------------------------------------------- host side
// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on the Legendre recurrence.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// psi_hat(d) = int psi(u) cos(2 pi d u / nfine) du over |u| <= w/2, for modes d = -(nmodes/2) ..
// (output index i <-> d = i - nmodes/2 for the image tables, d = i - (nmodes-1)/2 for K).
void nufft_psi_table(int nmodes, int nfine, int w, double beta, std::vector<double>& out) {
  std::vector<double> x, wt;
  gauss_legendre(4 * w + 40, x, wt);
  const int off = (nmodes % 2 == 1) ? (nmodes - 1) / 2 : nmodes / 2;
  out.resize(nmodes);
  for (int i = 0; i < nmodes; ++i) {
    const int d = i - off;
    double s = 0.0;
    for (size_t q = 0; q < x.size(); ++q) {
      const double u = 0.5 * w * x[q];
      const double z = x[q];
      const double t = 1.0 - z * z;
      const double psi = t > 0 ? exp(beta * (sqrt(t) - 1.0)) : 0.0;
      s += wt[q] * psi * cos(2.0 * M_PI * d * u / nfine);
    }
    out[i] = 0.5 * w * s;
  }
}

// Scratch carve-up (complex elements, FP64 worst case):
//   kernel spectrum:  tw[4N] | grid[(4N)^2] | tmp[(4N)^2]   (the 2N circulant FFT reuses grid);
//                     summed directly: tw[4N] | grid[(2N)^2] | tmp[(2N)^2] | cos/sin[n_angles]
//   back-projection:  tw[2N] | strengths[n_angles * n_det] | grid[(2N)^2] | tmp[(2N)^2]
// K by direct summation when the rows of the 4N NUFFT grid do not fit shared memory and are
// not a power of two (no in-place fallback): the 2560 side
static bool kernel_direct(int N) {
  const size_t nf = 4 * (size_t)N;
  return 2 * nf * sizeof(double2) > 200 * 1024 && (nf & (nf - 1)) != 0;
}

// complex elements of one back-projection batch on the grid of spreading configuration k:
// twiddles, strengths, grids, pruned transposes, sample-major strengths (kBackprojBatch wide)
static size_t backproject_elems(const tmbir_group& g, int k) {
  const size_t N = g.N, nf = spread_grid(k, g.N);
  const size_t rows = (size_t)g.n_angles * g.n_det;
  const size_t B = std::min(g.n_slices, kBackprojBatch);
  return nf + B * rows + B * nf * nf + B * N * nf + (size_t)kBackprojBatch * rows;
}
size_t setup_scratch_bytes(const tmbir_group& g) {
  const size_t N = g.N, nf_k = 4 * N, M = 2 * N, nf0 = spread_grid(0, g.N);
  const size_t k_elems = kernel_direct(g.N) ? nf_k + 2 * M * M + (size_t)g.n_angles : nf_k + 2 * nf_k * nf_k;
  // R*g in FP64 on grid 1; the FP32 back-projection of the direct operators on grid 0
  const size_t a_bytes = std::max(backproject_elems(g, 1) * sizeof(double2), backproject_elems(g, 0) * sizeof(float2));
  const size_t csr_build = (nf0 * nf0 + 2 * ((nf0 * nf0 + 2048) / 2048 + 1)) * sizeof(int);
  return std::max(std::max(std::max(k_elems * sizeof(double2), a_bytes), csr_build) + 256, forward_scratch_bytes(g));
}
size_t fbp_scratch_bytes(const tmbir_group& g) { return backproject_elems(g, 0) * sizeof(float2) + 256; }
size_t spread_nnz(const tmbir_group& g, int k) {
  return (size_t)g.n_angles * (g.n_det - 1) * kSpreadWidth[k] * kSpreadWidth[k];
}

// device twiddle tables for the setup FFTs (n up to 4N), carved from the front of the scratch
template <class C>
__global__ void k_twiddle(C* tw, int n) {
  using S = real_t<C>;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double sv, cv;
    sincospi(-2.0 * j / n, &sv, &cv);
    tw[j] = mkc((S)cv, (S)sv);
  }
}

// K(d) = (1/n_det) sum_a w_a D(e_a . d) summed directly, D(t) = sin(pi (n_det - 1) e / n_det) /
// sin(pi e / n_det) with e = t reduced to the nearest period of n_det, and n_det - 1 where the
// denominator vanishes; cs holds (cos, sin) of every angle, wts the weights w_a (nullptr: 1)
__global__ void k_angle_table(const double* __restrict__ angles, int na, double2* cs) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < na; a += gridDim.x * blockDim.x) {
    double sv, cv;
    sincos(angles[a], &sv, &cv);
    cs[a] = make_double2(cv, sv);
  }
}
__global__ void k_kernel_direct(const double2* __restrict__ cs, int na, int nd, int N, double* __restrict__ K,
                                const double* __restrict__ wts) {
  const int W = 2 * N - 1;
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < W * W; id += gridDim.x * blockDim.x) {
    const double dx = (double)(id % W - (N - 1)), dy = (double)(id / W - (N - 1));
    double sum = 0.0;
    for (int a = 0; a < na; ++a) {
      const double2 e2 = cs[a];
      const double t = dx * e2.x + dy * e2.y;
      const double e = t - (double)nd * rint(t / (double)nd);
      const double den = sinpi(e / (double)nd);
      const double D = den == 0.0 ? (double)(nd - 1) : sinpi((double)(nd - 1) * e / (double)nd) / den;
      sum += wts ? wts[a] * D : D;
    }
    K[id] = sum / (double)nd;
  }
}

static int circulant_spectrum(Ctx& c, int gi);

int build_kernel_spectrum(Ctx& c, int gi) {
  GroupDev& g = c.gdev[gi];
  cudaStream_t s = c.stream;
  const int N = g.N, nf = 4 * N, M = 2 * N;
  if (kernel_direct(N)) {
    double2* cs = reinterpret_cast<double2*>(c.scratch) + nf + 2 * (size_t)M * M;
    k_angle_table<<<(g.na + 255) / 256, 256, 0, s>>>(g.angles, g.na, cs);
    TMBIR_CHECK_LAUNCH();
    k_kernel_direct<<<152 * 16, 256, 0, s>>>(cs, g.na, g.nd, N, g.K, g.wts);
    TMBIR_CHECK_LAUNCH();
    return circulant_spectrum(c, gi);
  }
  double2* tw = reinterpret_cast<double2*>(c.scratch);
  double2* grid = tw + nf;
  double2* tmp = grid + (size_t)nf * nf;
  k_twiddle<double2><<<(nf + 255) / 256, 256, 0, s>>>(tw, nf);
  TMBIR_CHECK_LAUNCH();
  unsigned long long* fixed_grid = reinterpret_cast<unsigned long long*>(tmp);
  TMBIR_CUDA(cudaMemsetAsync(fixed_grid, 0, sizeof(unsigned long long) * nf * nf, s));
  {
    const size_t total = (size_t)g.na * (g.nd - 1);
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    k_spread_fixed<12><<<blocks, 256, 0, s>>>(g.angles, g.na, g.nd, nf, fixed_grid, c.nufft_beta64, g.wts);
    TMBIR_CHECK_LAUNCH();
  }
  k_fixed_to_complex<<<1024, 256, 0, s>>>(fixed_grid, grid, (size_t)nf * nf);
  TMBIR_CHECK_LAUNCH();
  if (int e = fft2_transposed(grid, tmp, nf, 1, +1, tw, s)) return e;
  k_deconv_K<<<1024, 256, 0, s>>>(tmp, nf, N, g.psiK, g.K);
  TMBIR_CHECK_LAUNCH();
  return circulant_spectrum(c, gi);
}

// real spectrum of the 2N x 2N circulant embedding of K, in the layout of pass 2
static int circulant_spectrum(Ctx& c, int gi) {
  GroupDev& g = c.gdev[gi];
  cudaStream_t s = c.stream;
  const int N = g.N, M = 2 * N;
  double2* tw = reinterpret_cast<double2*>(c.scratch);
  double2* grid = tw + 4 * (size_t)N;  // past the largest twiddle table
  k_twiddle<double2><<<(M + 255) / 256, 256, 0, s>>>(tw, M);
  TMBIR_CHECK_LAUNCH();
  double2* cg = grid;
  double2* ct = grid + (size_t)M * M;
  k_circulant<<<1024, 256, 0, s>>>(g.K, N, cg);
  TMBIR_CHECK_LAUNCH();
  if (int e = fft2_transposed(cg, ct, M, 1, -1, tw, s)) return e;
  k_chat_layout<<<1024, 256, 0, s>>>(ct, N, g.chat);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

int build_spread_matrix(Ctx& c, int gi) {
  GroupDev& g = c.gdev[gi];
  cudaStream_t s = c.stream;
  const size_t total = (size_t)g.na * (g.nd - 1);
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
  for (int k = 0; k < 2; ++k) {
    GroupDev::Spread& sp = g.sp[k];
    const int nf = sp.nf, ncells = nf * nf, W = kSpreadWidth[k];
    int* cursor = reinterpret_cast<int*>(c.scratch);
    int* sums = cursor + ncells;
    TMBIR_CUDA(cudaMemsetAsync(sp.ptr, 0, sizeof(int) * (ncells + 1), s));
    k_csr_count<<<blocks, 256, 0, s>>>(g.angles, g.na, g.nd, nf, W, sp.ptr);
    TMBIR_CHECK_LAUNCH();
    const int ntiles = (ncells + 1 + 2047) / 2048;
    k_scan_tiles<<<ntiles, 256, 0, s>>>(sp.ptr, ncells + 1, sums);
    TMBIR_CHECK_LAUNCH();
    k_scan_sums<<<1, 32, 0, s>>>(sums, ntiles);
    TMBIR_CHECK_LAUNCH();
    k_scan_add<<<1024, 256, 0, s>>>(sp.ptr, ncells + 1, sums);
    TMBIR_CHECK_LAUNCH();
    TMBIR_CUDA(cudaMemcpyAsync(cursor, sp.ptr, sizeof(int) * ncells, cudaMemcpyDeviceToDevice, s));
    k_csr_fill<<<blocks, 256, 0, s>>>(g.angles, g.na, g.nd, nf, W, spread_beta(k), cursor, sp.idx, sp.wt);
    TMBIR_CHECK_LAUNCH();
    k_csr_sort<<<(ncells + 255) / 256, 256, 0, s>>>(sp.ptr, ncells, sp.idx, sp.wt);
    TMBIR_CHECK_LAUNCH();
    if (k == 1) {  // R*g runs in double-word FP32: its weights as (hi, lo) pairs
      k_wt_to_df<<<1024, 256, 0, s>>>(sp.wt, spread_nnz(c.groups[gi], 1));
      TMBIR_CHECK_LAUNCH();
    }
  }
  return TMBIR_OK;
}

template <class C>
static int backproject_t(Ctx& c, int gi, const float* d_sino, float* d_out, bool ramp, float scale, char* scratch,
                         cudaStream_t s, bool local_out, const double* wts) {
  GroupDev& g = c.gdev[gi];
  // R*g in double-word FP32 on the 5N/4 grid, the FP32 back-projections on the 2N grid
  const GroupDev::Spread& sp = g.sp[sizeof(real_t<C>) == 8 ? 1 : 0];
  const int N = g.N, nf = sp.nf, nd = g.nd, na = g.na, ncells = nf * nf;
  const size_t rows = (size_t)na * nd;
  const int B = std::min(g.S, kBackprojBatch);
  C* tw = reinterpret_cast<C*>(scratch);
  C* strengths = tw + nf;
  C* grid = strengths + (size_t)B * rows;
  C* tmp = grid + (size_t)B * ncells;
  C* strengths_t = tmp + (size_t)B * N * nf;  // [rows][kBackprojBatch]
  for (int b0 = 0; b0 < g.S; b0 += B) {
    const int nb = std::min(B, g.S - b0);
    const float* sino_b = d_sino + g.sino_off + (size_t)b0 * rows;
    // radial 1D transform of every projection: G(a, k)
    k_prepare_rows<C><<<(int)std::min<size_t>((size_t)nb * na, 4096), 256, 2 * nd * sizeof(float), s>>>(
        sino_b, nd, (size_t)nb * na, ramp ? 1 : 0, strengths);
    TMBIR_CHECK_LAUNCH();
    k_twiddle<C><<<(nd + 255) / 256, 256, 0, s>>>(tw, nd);
    TMBIR_CHECK_LAUNCH();
    if (int e = fft_rows(strengths, nd, nb * na, +1, tw, s)) return e;
    constexpr int PB = kBackprojBatch / 2;  // slice pairs per batch
    const int np = (nb + 1) / 2;
    k_strength_pack<PB, C><<<1024, 256, 0, s>>>(strengths, nd, rows, nb, strengths_t, wts);
    TMBIR_CHECK_LAUNCH();
    k_csr_gather<PB, C><<<(ncells + 255) / 256, 256, 0, s>>>(sp.ptr, sp.idx, sp.wt, ncells, strengths_t,
                                                              grid, np);
    TMBIR_CHECK_LAUNCH();
    k_twiddle<C><<<(nf + 255) / 256, 256, 0, s>>>(tw, nf);
    TMBIR_CHECK_LAUNCH();
    // 2D transform of the pair grids with the output pruned to the N x N image modes
    if (int e = fft_rows(grid, nf, np * nf, -1, tw, s)) return e;
    {
      dim3 gr((N + 31) / 32, (nf + 31) / 32, np), bl(32, 8);
      k_transpose_prune<C><<<gr, bl, 0, s>>>(grid, tmp, nf, N);
      TMBIR_CHECK_LAUNCH();
    }
    if (int e = fft_rows(tmp, nf, np * N, -1, tw, s)) return e;
    {
      dim3 gr((N + 31) / 32, (N + 31) / 32, np), bl(32, 8);
      k_deconv_pruned<C><<<gr, bl, 0, s>>>(tmp, nf, N, nb, sp.psi, scale,
                                           d_out + (local_out ? 0 : g.img_off) + (size_t)b0 * N * N);
    }
    TMBIR_CHECK_LAUNCH();
  }
  return TMBIR_OK;
}

int backproject(Ctx& c, int gi, const float* d_sino, float* d_out, bool ramp, bool fp64, char* scratch,
                cudaStream_t s, bool local_out, bool weighted) {
  const GroupDev& g = c.gdev[gi];
  const float scale = ramp ? (float)(g.span / g.na) : 1.0f;
  const double* wts = weighted ? g.wts : nullptr;
  if (!scratch) scratch = c.scratch;
  if (!s) s = c.stream;
  if (fp64) return backproject_t<dfc>(c, gi, d_sino, d_out, ramp, scale, scratch, s, local_out, wts);
  return backproject_t<float2>(c, gi, d_sino, d_out, ramp, scale, scratch, s, local_out, wts);
}

int half_sumsq(Ctx& c, const float* p, size_t n, double* d_out, cudaStream_t s, const double* wts, int na, int nd) {
  if (!s) s = c.stream;
  double* part = reinterpret_cast<double*>(c.scratch);
  k_sumsq_blocks<<<1024, 256, 0, s>>>(p, n, part, wts, na, nd);
  TMBIR_CHECK_LAUNCH();
  k_sum_half<<<1, 256, 0, s>>>(part, 1024, d_out);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

// ---------------------------------------------------------------- forward projection (type-2 NUFFT)
// R x(a, m) = (1/n_det) sum_k exp(-2 pi i k s_m / n_det) xhat(xi_{a,k}),
// xhat(xi) = sum_x x(x) exp(+2 pi i xi . x)  (Eqs. 3-4, the adjoint of the back-projection):
// divide the image by the kernel's Fourier transform, place it on the 2N x 2N periodic grid,
// FFT with the + sign, interpolate at the polar samples with the spreading kernel (width
// kSpreadW), then the radial 1D transform.  FP32; two slices share one complex grid (the
// result of a real image pair is R x_{2p} + i R x_{2p+1}).

// grid[p][row'][col'] = (x_{2p} + i x_{2p+1})[r][c] / (psi[c] psi[r]) at row' = (r - N/2) mod nf,
// col' = (c - N/2) mod nf, zero elsewhere
__global__ void k_pad_deconv_pairs(const float* __restrict__ x, int N, int nf, int nb, const double* __restrict__ psi,
                                   float2* __restrict__ grid) {
  const int np = (nb + 1) / 2;
  const size_t cells = (size_t)nf * nf, total = (size_t)np * cells, plane = (size_t)N * N;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(id / cells);
    const int cell = (int)(id % cells), rp = cell / nf, cp = cell % nf;
    const int r = (rp + N / 2) % nf, c = (cp + N / 2) % nf;
    float2 v = make_float2(0.f, 0.f);
    if (r < N && c < N) {
      const float inv = (float)(1.0 / (psi[c] * psi[r]));
      const size_t o = (size_t)r * N + c;
      v.x = x[(size_t)(2 * p) * plane + o] * inv;
      if (2 * p + 1 < nb) v.y = x[(size_t)(2 * p + 1) * plane + o] * inv;
    }
    grid[id] = v;
  }
}

__device__ __forceinline__ float es_kernel_f(float z, float beta) {  // z in [-1, 1]
  const float t = 1.f - z * z;
  return t > 0.f ? expf(beta * (sqrtf(t) - 1.f)) : 0.f;
}

// rows[p][a][k mod n_det] = (-1)^k / n_det * sum_l psi(u - l) F_p[l] for |k| <= n_det/2 - 1 (0 at
// the Nyquist index), F transposed ([lx][ly]); one thread per sample, all pairs of the batch
template <int W, int PB>
__global__ void k_interp_pairs(const float2* __restrict__ F, const double* __restrict__ angles, int na, int nd, int nf,
                               float beta, int np, float2* __restrict__ rows) {
  const size_t total = (size_t)na * nd, cells = (size_t)nf * nf;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const int kk = (int)(id % nd), a = (int)(id / nd);
    float2 acc[PB];
#pragma unroll
    for (int p = 0; p < PB; ++p) acc[p] = make_float2(0.f, 0.f);
    if (kk != nd / 2) {
      const int k = kk < nd / 2 ? kk : kk - nd;
      double sa, ca;
      sincos(angles[a], &sa, &ca);
      const double ux = (double)k * ca * nf / nd, uy = (double)k * sa * nf / nd;
      const int lx0 = (int)ceil(ux - 0.5 * W), ly0 = (int)ceil(uy - 0.5 * W);
      float wx[W], wy[W];
#pragma unroll
      for (int j = 0; j < W; ++j) {
        wx[j] = es_kernel_f((float)((2.0 * (lx0 + j - ux)) / W), beta);
        wy[j] = es_kernel_f((float)((2.0 * (ly0 + j - uy)) / W), beta);
      }
#pragma unroll 1
      for (int jx = 0; jx < W; ++jx) {
        const int lx = (lx0 + jx + nf) % nf;
#pragma unroll
        for (int p = 0; p < PB; ++p) {
          if (p < np) {
            const float2* col = F + (size_t)p * cells + (size_t)lx * nf;
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int jy = 0; jy < W; ++jy) {
              const float2 v = col[(ly0 + jy + nf) % nf];
              s.x = fmaf(wy[jy], v.x, s.x);
              s.y = fmaf(wy[jy], v.y, s.y);
            }
            acc[p].x = fmaf(wx[jx], s.x, acc[p].x);
            acc[p].y = fmaf(wx[jx], s.y, acc[p].y);
          }
        }
      }
      const float sg = (k & 1) ? -1.f / nd : 1.f / nd;
#pragma unroll
      for (int p = 0; p < PB; ++p) acc[p] = make_float2(acc[p].x * sg, acc[p].y * sg);
    }
#pragma unroll
    for (int p = 0; p < PB; ++p)
      if (p < np) rows[(size_t)p * total + id] = acc[p];
  }
}

// sino[b][a][m] = Re (b even) or Im (b odd) of rows[b / 2][a][m]
__global__ void k_unpack_pairs(const float2* __restrict__ rows, size_t per_pair, int nb, float* __restrict__ sino) {
  const size_t total = (size_t)nb * per_pair;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(id / per_pair);
    const float2 v = rows[(size_t)(b / 2) * per_pair + id % per_pair];
    sino[id] = (b & 1) ? v.y : v.x;
  }
}

size_t forward_scratch_bytes(const tmbir_group& g) {
  const size_t nf = spread_grid(0, g.N), np = (std::min(g.n_slices, kBackprojBatch) + 1) / 2;
  return (nf + g.n_det + 2 * np * nf * nf + np * (size_t)g.n_angles * g.n_det) * sizeof(float2) + 256;
}

int forward_project(Ctx& c, int gi, const float* d_x, float* d_sino, cudaStream_t s) {
  GroupDev& g = c.gdev[gi];
  if (!s) s = c.stream;
  const GroupDev::Spread& sp = g.sp[0];  // FP32: the 2N grid
  const int N = g.N, nf = sp.nf, nd = g.nd, na = g.na;
  const size_t cells = (size_t)nf * nf, rows = (size_t)na * nd;
  const int B = std::min(g.S, kBackprojBatch);
  constexpr int PB = kBackprojBatch / 2;
  if (forward_scratch_bytes(c.groups[gi]) > c.scratch_bytes)
    return set_error(TMBIR_ERR_WORKSPACE, "forward projection: setup scratch too small");
  float2* tw_f = reinterpret_cast<float2*>(c.scratch);
  float2* tw_d = tw_f + nf;
  float2* grid = tw_d + nd;
  float2* tmp = grid + (size_t)PB * cells;
  float2* prow = tmp + (size_t)PB * cells;
  k_twiddle<float2><<<(nf + 255) / 256, 256, 0, s>>>(tw_f, nf);
  TMBIR_CHECK_LAUNCH();
  k_twiddle<float2><<<(nd + 255) / 256, 256, 0, s>>>(tw_d, nd);
  TMBIR_CHECK_LAUNCH();
  for (int b0 = 0; b0 < g.S; b0 += B) {
    const int nb = std::min(B, g.S - b0), np = (nb + 1) / 2;
    k_pad_deconv_pairs<<<1024, 256, 0, s>>>(d_x + g.img_off + (size_t)b0 * N * N, N, nf, nb, sp.psi, grid);
    TMBIR_CHECK_LAUNCH();
    if (int e = fft2_transposed(grid, tmp, nf, np, +1, tw_f, s)) return e;
    k_interp_pairs<kSpreadWidth[0], PB><<<(int)std::min<size_t>((rows + 255) / 256, 152 * 16), 256, 0, s>>>(
        tmp, g.angles, na, nd, nf, (float)spread_beta(0), np, prow);
    TMBIR_CHECK_LAUNCH();
    if (int e = fft_rows(prow, nd, np * na, -1, tw_d, s)) return e;
    k_unpack_pairs<<<1024, 256, 0, s>>>(prow, rows, nb, d_sino + g.sino_off + (size_t)b0 * rows);
    TMBIR_CHECK_LAUNCH();
  }
  return TMBIR_OK;
}

// d_sino -= d_g over one group (the residual R x - g)
__global__ void k_sub_inplace(float* __restrict__ a, const float* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] -= b[i];
}
int residual(Ctx& c, int gi, float* d_rx, const float* d_g, cudaStream_t s) {
  const GroupDev& g = c.gdev[gi];
  if (!s) s = c.stream;
  const size_t n = (size_t)g.S * g.na * g.nd;
  k_sub_inplace<<<1024, 256, 0, s>>>(d_rx + g.sino_off, d_g + g.sino_off, n);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

int group_gtg(Ctx& c, int gi, const float* d_sino) {
  const GroupDev& g = c.gdev[gi];
  const float* p = d_sino + g.sino_off;
  double* part = reinterpret_cast<double*>(c.scratch);
  k_sumsq_blocks<<<1024, 256, 0, c.stream>>>(p, (size_t)g.S * g.na * g.nd, part, g.wts, g.na, g.nd);
  TMBIR_CHECK_LAUNCH();
  k_sum_half<<<1, 256, 0, c.stream>>>(part, 1024, g.gtg);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

// lambda_max(R*R) of a group: 100 power steps on one slice from the all-ones image
int power_iteration(Ctx& c, int gi, int steps) {
  GroupDev g = c.gdev[gi];
  cudaStream_t s = c.stream;
  const size_t n = (size_t)g.N * g.N;
  // one-slice view of the group; images live in the two iterate buffers
  g.S = 1;
  g.slice0 = 0;
  g.img_off = 0;
  float* v = c.xbuf[0];
  float* w = c.xbuf[1];
  k_fill<<<256, 256, 0, s>>>(v, n, (float)(1.0 / g.N));
  TMBIR_CHECK_LAUNCH();
  PriorC pc{};
  for (int it = 0; it < steps; ++it) {
    StepArgs a{};
    a.x = v;
    a.xprev = v;
    a.beta = 0.f;
    a.out = w;
    a.st = nullptr;
    if (int e = launch_convolution(g, a, Pass3Mode::Apply, pc, s)) return e;
    if (int e = launch_pass3(g, a, Pass3Mode::Apply, pc, c.partials, 0, s, false, 2)) return e;
    if (int e = launch_sum_partials(c.partials, blocks_pass3(g), c.dscal, s)) return e;
    k_normalize<<<256, 256, 0, s>>>(w, v, n, c.dscal, g.lam_max);
    TMBIR_CHECK_LAUNCH();
  }
  return TMBIR_OK;
}

}  // namespace tmbir
