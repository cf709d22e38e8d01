// Reductions, the optimiser state update and the size dispatch of the Toeplitz passes.
// The passes themselves live in toeplitz_kernels.cuh (instantiated per image side by
// toeplitz_inst.cu).
#include "fft.cuh"
#include "internal.h"

namespace tmbir {

bool supported_N(int N) {
  return N == 64 || N == 128 || N == 256 || N == 512 || N == 1024 || N == 2048 || N == 1536 || N == 2560;
}
bool block_fft_N(int N) { return N == 1536 || N == 2560; }

void fft_shape(int N, int* T, int* P) {
  switch (N) {
    case 64: *T = 8; *P = 8; break;
    case 128: *T = 8; *P = 16; break;
    case 256: *T = 16; *P = 16; break;
    case 512: *T = 16; *P = 32; break;
    case 1024: *T = 32; *P = 32; break;
    case 2048: *T = 32; *P = 64; break;
    default: *T = 32; *P = N / 32; break;  // 1536, 2560: rows of the block-FFT passes
  }
}

#define TMBIR_DECL_N(N)                                                                                     \
  int pass1_##N(const GroupDev* gs, int n, const StepArgs& a, bool bf16, cudaStream_t s);                   \
  int pass2_##N(const GroupDev* gs, int n, const IterState* st, bool bf16, cudaStream_t s);                 \
  int pass3_##N(const GroupDev* gs, int n, const StepArgs& a, Pass3Mode m, const PriorC& pc, double* partials, \
                int off, bool bf16, int part, cudaStream_t s);
TMBIR_DECL_N(64)
TMBIR_DECL_N(128)
TMBIR_DECL_N(256)
TMBIR_DECL_N(512)
TMBIR_DECL_N(1024)
TMBIR_DECL_N(2048)
TMBIR_DECL_N(1536)
TMBIR_DECL_N(2560)
#undef TMBIR_DECL_N

// ---------------------------------------------------------------- reductions and state update
__device__ void reduce_blocks(const double* partials, int nblocks, double* outv) {
  __shared__ double sh[512];
  for (int j = 0; j < kParts; ++j) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(size_t)b * kParts + j];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) outv[j] = sh[0];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(512) k_sum_partials(const double* partials, int nblocks, double* out) {
  reduce_blocks(partials, nblocks, out);
}

// Reduces the partial sums of one iteration and advances the optimiser state (Eq. 6 with the
// restart test): per group its momentum sequence and restart decision (the group's blocks are
// the rows gb.off[g] .. gb.off[g + 1] of the partials, reduced in the same order as in a context
// of that group alone), over all groups the objective, the stop rule, the storage phase and the
// buffer rotation.  Inside a device-driven graph loop it also sets the loop's condition: 0 once
// the run is done (every path sets it, so the loop always ends by max_iter).
__global__ void __launch_bounds__(512) k_finalize(IterState* st, GroupMom* gm, const double* partials, GroupBlocks gb,
                                                  double* log, cudaGraphConditionalHandle cond, int use_cond,
                                                  int trip_launches) {
  __shared__ double S[kParts];
  __shared__ double tot[4];  // F, <G, x_new - x>, G.G, restarts
  if (st->done) {
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
    return;
  }
  if (threadIdx.x == 0) tot[0] = tot[1] = tot[2] = tot[3] = 0.0;
  const int k = st->k;
  for (int g = 0; g < gb.n; ++g) {
    reduce_blocks(partials + (size_t)gb.off[g] * kParts, gb.off[g + 1] - gb.off[g], S);
    if (threadIdx.x == 0) {
      GroupMom& m = gm[g];
      const double yz = S[0], yatg = S[1], phi = S[2], gdx = S[3], gg = S[4];
      const double F = 0.5 * yz - yatg + m.gtg_half + st->lambda * phi;
      // gradient restart: <grad F(y_k), x_{k+1} - x_k> > 0; function restart: F(y_k) > F(y_{k-1})
      const bool restart = (st->restart_mode == TMBIR_RESTART_GRADIENT && gdx > 0.0) ||
                           (st->restart_mode == TMBIR_RESTART_FUNCTION && k > 0 && F > m.prev_F);
      m.prev_F = F;
      const double tn = restart ? 1.0 : 0.5 * (1.0 + sqrt(1.0 + 4.0 * m.t * m.t));
      const double tnn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tn * tn));
      m.beta = (tn - 1.0) / tnn;
      m.t = tn;
      m.restarts += restart ? 1 : 0;
      tot[0] += F;
      tot[1] += gdx;
      tot[2] += gg;
      tot[3] += restart ? 1.0 : 0.0;
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double F = tot[0], gdx = tot[1], gg = tot[2];
  if (k < st->log_cap) {
    log[4 * k + 0] = F;
    log[4 * k + 1] = gdx;
    log[4 * k + 2] = tot[3];  // groups that restarted (0 or 1 for one group)
    log[4 * k + 3] = gg;
  }
  st->restarts += (int)tot[3];
  st->prev_F = F;
  st->k = k + 1;
  st->cur = (st->cur + 1) % 3;
  st->last_F = F;
  st->last_dot = gdx;
  st->last_gg = gg;
  double gap = 0.0;
  if (st->Fref == st->Fref && st->F0 != st->Fref) gap = (F - st->Fref) / (st->F0 - st->Fref);
  st->last_gap = gap;
  // BF16 -> FP32 refinement: later iterations store the spectrum in FP32
  if (st->bf16 && st->refine_gap > 0.0 && gap <= st->refine_gap) st->bf16 = 0;
  if (!isfinite(F) || !isfinite(gdx) || !isfinite(gg)) {
    st->status = TMBIR_ERR_NONFINITE;
    st->done = 1;
  }
  if (k + 1 >= st->max_iter) st->done = 1;
  if (st->gap_tol > 0.0 && gap <= st->gap_tol) st->done = 1;
  if (use_cond) {
    // loop kind 1 runs to the end of the run; kind 2 (the BF16 loop) also ends at the switch
    st->graph_launches += trip_launches;
    cudaGraphSetConditional(cond, (st->done || (use_cond == 2 && !st->bf16)) ? 0 : 1);
  }
}

#define TMBIR_DISPATCH_N(N_, FN, ...)                               \
  switch (N_) {                                                     \
    case 64: return FN##64(__VA_ARGS__);                            \
    case 128: return FN##128(__VA_ARGS__);                          \
    case 256: return FN##256(__VA_ARGS__);                          \
    case 512: return FN##512(__VA_ARGS__);                          \
    case 1024: return FN##1024(__VA_ARGS__);                        \
    case 2048: return FN##2048(__VA_ARGS__);                        \
    case 1536: return FN##1536(__VA_ARGS__);                        \
    case 2560: return FN##2560(__VA_ARGS__);                        \
    default: return set_error(TMBIR_ERR_SHAPE, "unsupported N");    \
  }

int launch_pass1(const GroupDev& g, const StepArgs& a, cudaStream_t s, bool bf16) {
  TMBIR_DISPATCH_N(g.N, pass1_, &g, 1, a, bf16, s);
}
int launch_pass2(const GroupDev& g, const IterState* st, cudaStream_t s, bool bf16) {
  TMBIR_DISPATCH_N(g.N, pass2_, &g, 1, st, bf16, s);
}
int launch_pass3(const GroupDev& g, const StepArgs& a, Pass3Mode m, const PriorC& pc, double* partials, int off,
                 cudaStream_t s, bool bf16, int part) {
  TMBIR_DISPATCH_N(g.N, pass3_, &g, 1, a, m, pc, partials, off, bf16, part, s);
}
bool launch_set_ok(const GroupDev& first, const GroupDev& g) {
  return g.N == first.N && g.rb1 == first.rb1 && g.rb3 == first.rb3 && spec_chunk(g) == g.S &&
         spec_chunk(first) == first.S;
}
static int pass1_set(const GroupDev* gs, int n, const StepArgs& a, cudaStream_t s, bool bf16) {
  TMBIR_DISPATCH_N(gs[0].N, pass1_, gs, n, a, bf16, s);
}
static int pass2_set(const GroupDev* gs, int n, const IterState* st, cudaStream_t s, bool bf16) {
  TMBIR_DISPATCH_N(gs[0].N, pass2_, gs, n, st, bf16, s);
}
static int pass3_set(const GroupDev* gs, int n, const StepArgs& a, const PriorC& pc, double* partials, int off,
                     cudaStream_t s, bool bf16, int part) {
  TMBIR_DISPATCH_N(gs[0].N, pass3_, gs, n, a, Pass3Mode::Iterate, pc, partials, off, bf16, part, s);
}
int launch_passes_set(const GroupDev* gs, int n, const StepArgs& a, const PriorC& pc, double* partials,
                      int block_offset, cudaStream_t s, bool bf16) {
  if (n < 1 || n > kMergeMax) return set_error(TMBIR_ERR_ARG, "group set size");
  for (int i = 1; i < n; ++i)
    if (!launch_set_ok(gs[0], gs[i])) return set_error(TMBIR_ERR_ARG, "groups of one launch must share its shape");
  if (int e = pass1_set(gs, n, a, s, bf16)) return e;
  if (int e = pass2_set(gs, n, a.st, s, bf16)) return e;
  if (int e = pass3_set(gs, n, a, pc, nullptr, 0, s, bf16, 1)) return e;
  return pass3_set(gs, n, a, pc, partials, block_offset, s, bf16, 2);
}
GroupDev chunk_view(const GroupDev& g, int c0, int n) {
  GroupDev v = g;
  const size_t off = (size_t)c0 * g.N * g.N;
  v.S = n;
  v.slice0 = g.slice0 + c0;
  v.img_off = g.img_off + off;
  if (g.kz) v.kz = g.kz + off;
  return v;
}
int launch_convolution(const GroupDev& g, const StepArgs& a, Pass3Mode m, const PriorC& pc, cudaStream_t s,
                       bool bf16) {
  const int sc = spec_chunk(g);
  for (int c0 = 0; c0 < g.S; c0 += sc) {
    const GroupDev v = chunk_view(g, c0, g.S - c0 < sc ? g.S - c0 : sc);
    if (int e = launch_pass1(v, a, s, bf16)) return e;
    if (int e = launch_pass2(v, a.st, s, bf16)) return e;
    if (int e = launch_pass3(v, a, m, pc, nullptr, 0, s, bf16, 1)) return e;
  }
  return TMBIR_OK;
}
int conv_launches(const GroupDev& g) {
  const int sc = spec_chunk(g);
  return 3 * ((g.S + sc - 1) / sc);
}

int blocks_pass3(const GroupDev& g) {
  const int nb = pass3_row_blocks(g.N);
  const int zc = pass3_zc(g, nb);
  return nb * ((pass3_slices(g) + zc - 1) / zc);
}
int max_blocks_pass3(const GroupDev& g) { return pass3_row_blocks(g.N) * g.S; }

int launch_finalize(IterState* st, GroupMom* gm, const double* partials, const GroupBlocks& gb, double* log,
                    cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond, int trip_launches) {
  k_finalize<<<1, 512, 0, s>>>(st, gm, partials, gb, log, cond, use_cond, trip_launches);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}
int launch_sum_partials(const double* partials, int nblocks, double* out, cudaStream_t s) {
  k_sum_partials<<<1, 512, 0, s>>>(partials, nblocks, out);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

}  // namespace tmbir
