// Internal declarations shared by the translation units of libtmbir.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tmbir.h"

namespace tmbir {

// Device-resident optimiser state, advanced by the finalize kernel once per iteration.  The
// momentum, step constant and restart test are per geometry group (GroupMom): groups are
// independent problems; the stop rule, the storage phase and the buffer rotation are shared.
struct IterState {
  double t;         // unused (per group: GroupMom)
  double beta;      // unused (per group: GroupMom)
  double L, invL;   // step constant of the first group (reported in the stats)
  double lambda;    // prior weight
  double gtg_half;  // 1/2 g.g summed over all groups
  double F0, Fref, gap_tol;
  double last_F, last_gap, last_gg, last_dot;
  int k;            // iterations completed
  int max_iter;
  int restarts;
  int cur;          // xbuf[cur] = x_k, xbuf[(cur+2)%3] = x_{k-1}, xbuf[(cur+1)%3] = x_{k+1}
  int done;
  int status;
  int restart_mode;
  int log_cap;
  double prev_F;             // F(y_{k-1}), for the function-value restart
  int bf16;                  // 1 while the iterations store the spectrum in BF16
  double refine_gap;         // BF16 -> FP32 switch: gap <= refine_gap (with F_ref), or F(y_k) > F(y_{k-1})
  long long graph_launches;  // kernels run by device-driven graph trips, cumulative (zeroed at workspace binding)
};

// Fast-gradient state of one geometry group (Sec. 2, Eq. 6 with restart): its own step
// constant, momentum sequence and restart test, as if the group were reconstructed alone.
struct GroupMom {
  double t;         // momentum sequence t_k
  double beta;      // beta_k used by the current iteration
  double L, invL;   // step constant
  double prev_F;    // F_g(y_{k-1}), for the function-value restart
  double gtg_half;  // 1/2 g.g of the group
  int restarts;
  int pad;
};
constexpr int kMaxGroups = 64;
// First partial-sum row of each group's pass-3b blocks (off[n] = total), passed by value.
struct GroupBlocks {
  int n;
  int off[kMaxGroups + 1];
};

// Number of FP64 partial sums each reducing block writes.
constexpr int kParts = 6;  // y.z, y.atg, Phi(y), <G, x_new - x>, G.G, z.z
constexpr int kLogCap = 1 << 16;
// checkpoint layout: the iteration state in the first kStateHeader bytes, then x_{k-1}
constexpr size_t kStateHeader = 256;
static_assert(sizeof(IterState) <= kStateHeader, "checkpoint header too small");
// checkpoint bytes before x_{k-1}: the iteration state, then the groups' momentum states
inline size_t state_header_bytes(int n_groups) {
  return kStateHeader + ((size_t)n_groups * sizeof(GroupMom) + 255) / 256 * 256;
}

// qGGMRF constants in the form the kernels use.
struct PriorC {
  float p, q, qp;        // exponents and q - p
  float inv_csig;        // 1 / (c sigma)
  float inv_sig;         // 1 / sigma
  float inv_sig2;        // 1 / sigma^2
  float lam;             // lambda
  float wf, we, wc;      // face / edge / corner neighbour weights (sum of the 26 is 1)
  float l2_inv_csig;     // log2(1 / (c sigma))
  float qp_l2_inv_csig;  // (q - p) log2(1 / (c sigma))
  float l2_inv_sig;      // log2(1 / sigma)
  int q_is_2;
  int nonneg;            // project each iterate onto x >= 0
};

// One geometry group as the kernels see it (device pointers into the workspace).
struct GroupDev {
  int N, nd, na, S;
  int slice0;          // first slice of the group in the stacked arrays
  size_t img_off;      // first element of the group in the stacked image arrays
  size_t sino_off;     // first element of the group in the stacked sinogram
  float span;
  // Toeplitz operator
  float* chat;         // [N+1][2][N] real spectrum, even/odd rows of the 2N grid, scaled by 1/(2N)^2
  float2* twN;         // [P][T] exp(-2 pi i t k / N) for the row/column group FFT
  float2* twM;         // [N] exp(-2 pi i n / 2N)
  float2* spec;        // [S][N+1][N] intermediate spectra
  // setup
  double* angles;      // [na]
  double* K;           // [(2N-1)^2] point-spread kernel
  double* psiK;        // [2N-1] deconvolution factors for K (fine grid 4N)

  const double* wts;   // [na] per-angle weights of the data term (nullptr: all 1)
  double* lam_max;     // device scalar
  double* gtg;         // device scalar (1/2 g.g of the group)
  // sparse spreading operators (geometry only): sp[0] for the FP32 paths, sp[1] for R*g in FP64
  struct Spread {
    int nf;            // periodic grid side
    double* psi;       // [N] deconvolution factors (the kernel's Fourier transform at the image modes)
    int* ptr;          // [nf^2 + 1] rows of grid cells
    int* idx;          // [nnz] strength index a * n_det + (k mod n_det)
    double* wt;        // [nnz] kernel weight
  } sp[2];
  float* kz;           // [S][N][N] K (*) y between passes 3a and 3b
  int zc;              // slices each pass-3 block marches through (0: the default rule)
  // pass 3b's slice range [zlo, zlo + zn) (zn = 0: all S slices); the slices outside it are
  // neighbours only (the halo of a slab of a larger volume)
  int zlo, zn;
  int sc;              // slices per spectrum chunk of passes 1, 2, 3a (0: the default rule)
  int rb1, rb3;        // rows per block of passes 1 and 3a where a side has variants (0: default)
};

// Up to kMergeMax consecutive groups of one image side that one launch of a pass covers: block
// b of the launch belongs to the group i with boff[i] <= b < boff[i + 1].  Kernels take it as a
// __grid_constant__ parameter, so the per-block group lookup reads the parameter bank in place.
constexpr int kMergeMax = 8;
struct GroupSet {
  int n;
  int boff[kMergeMax + 1];
  GroupDev g[kMergeMax];
#ifdef __CUDACC__
  // the group of this block, and the block's index within that group (MULTI false: a set of one
  // group, whose fields the kernel then reads at fixed parameter offsets)
  template <bool MULTI = true>
  __device__ __forceinline__ int pick(int& bid) const {
    if constexpr (!MULTI) {
      bid = (int)blockIdx.x;
      return 0;
    }
    int i = 0;
    while (i + 1 < n && (int)blockIdx.x >= boff[i + 1]) ++i;
    bid = (int)blockIdx.x - boff[i];
    return i;
  }
#endif
};

// Passes 1, 2 and 3a may run in chunks of slices (a chunk's half spectra can then stay in L2
// between the three passes).  Measured on GB300 at 64 x 1024^2 the whole group in one chunk is
// fastest (the shorter launches lose more to launch gaps and partial last waves than L2 reuse
// saves), so that is the default; tmbir_autotune tries chunks of 4, 8 and 16 slices too.
inline int spec_chunk(const GroupDev& g) { return g.sc > 0 && g.sc < g.S ? g.sc : g.S; }

// The two spreading configurations of the back-projection (exponential-of-semicircle kernel,
// relative error of R* about 1e-9 / 1e-8):
//   0, the FP32 paths (FBP start, forward and adjoint projections): a 2N x 2N grid, width 10,
//      beta 2.30 per unit width;
//   1, R*g in FP64: a 5N/4 x 5N/4 grid (2^a 3^b 5^c for every supported side), width 14,
//      beta = 0.97 pi (1 - 1/(2 * 1.25)) per unit width.  The smaller grid cuts the FP64 grid
//      FFTs, which dominate the setup, to 0.37x for 1.96x the sparse gather; dividing by the
//      kernel's Fourier transform amplifies rounding towards the image corners (up to ~5e5 at
//      1.25, 13 at 2), harmless in FP64 but not in FP32, hence two configurations.
constexpr int kSpreadWidth[2] = {10, 14};
inline int spread_grid(int k, int N) { return k ? N * 5 / 4 : 2 * N; }
inline double spread_beta(int k) { return k ? 0.97 * 3.14159265358979323846 * (1.0 - 1.0 / 2.5) * 14 : 2.30 * 10; }
constexpr int kBackprojBatch = 8;  // slices per back-projection batch

struct Ctx {
  cudaStream_t stream = nullptr;
  std::vector<tmbir_group> groups;
  std::vector<std::vector<double>> angles;
  std::vector<GroupDev> gdev;
  // host copies of the NUFFT deconvolution tables (uploaded at set_workspace)
  std::vector<std::vector<double>> psiK_h, psiS_h[2];
  double nufft_beta64 = 0;
  std::vector<std::vector<double>> weights;  // per-angle data-term weights per group (empty: all 1)
  std::vector<bool> geom_ready;    // K, its spectrum and lambda_max built
  std::vector<bool> spread_ready;  // sparse spreading matrix built
  size_t total_voxels = 0, total_sino = 0;
  int total_slices = 0;
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0, ws_need = 0;
  IterState* state = nullptr;
  GroupMom* gmom = nullptr;    // [n_groups]
  double* partials = nullptr;  // [max_blocks][kParts]
  int max_blocks = 0;
  double* log = nullptr;       // [kLogCap][4]
  float* xbuf[2] = {nullptr, nullptr};
  char* scratch = nullptr;     // setup scratch (aliases nothing used across calls)
  size_t scratch_bytes = 0;
  double* dscal = nullptr;     // small FP64 device scalars [64]
  bool operator_built = false;
  int last_iters = 0;
  // layout offsets computed at set_geometry
  std::vector<size_t> off_chat, off_twN, off_twM, off_spec, off_kz, off_ang, off_K, off_psiK, off_lam, off_gtg, off_wts;
  std::vector<size_t> off_sp_psi[2], off_sp_ptr[2], off_sp_idx[2], off_sp_wt[2];
  size_t off_state = 0, off_gmom = 0, off_partials = 0, off_log = 0, off_xbuf0 = 0, off_xbuf1 = 0, off_scratch = 0, off_dscal = 0;
  size_t off_fbp_scratch = 0;
  char* fbp_scratch = nullptr;  // FP32 back-projection scratch, separate so FBP can overlap R*g
  float* sino_tmp = nullptr;    // a sinogram of the whole batch: R x and the residual of the direct gradient
  size_t off_sino_tmp = 0;
  cudaStream_t aux = nullptr;   // second stream for the overlapped FBP (created on first use)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // host volumes: copy-in and copy-out streams beside the context stream, events per buffer set
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  cudaEvent_t ev_start = nullptr;
  // CUDA graph cache for reconstruct
  cudaGraphExec_t graph_exec = nullptr;
  const float* graph_atg = nullptr;
  float* graph_x = nullptr;
  PriorC graph_prior{};
  int graph_kind = 0;
  bool state_ready = false;  // the iteration state holds a finished run (or an imported one)  // 1: one FP32 loop; 2: BF16 loop only; 3: BF16 loop then FP32 loop
};

// tracing -------------------------------------------------------------------
// An NVTX range around each C-ABI call, visible to Nsight tools when one is attached (the
// header-only NVTX API costs a branch otherwise).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
#define TMBIR_TRACE(name) ::tmbir::TraceRange tmbir_trace_range_(name)

// error handling ------------------------------------------------------------
int set_error(int code, const std::string& msg);
#define TMBIR_CUDA(call)                                                                    \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return ::tmbir::set_error(TMBIR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
// kernels launched by the library in this process (graph replays add their kernel nodes)
extern long long g_launches;
#define TMBIR_CHECK_LAUNCH()             \
  do {                                   \
    TMBIR_CUDA(cudaGetLastError());      \
    __atomic_add_fetch(&::tmbir::g_launches, 1, __ATOMIC_RELAXED); \
  } while (0)

// toeplitz.cu ---------------------------------------------------------------
enum class Pass3Mode { Apply = 0, Gradient = 1, Step = 2, Iterate = 3, Objective = 4 };

struct StepArgs {
  const float* x;       // x_k (or the image for apply/gradient/objective)
  const float* xprev;   // x_{k-1} (== x when beta = 0)
  float beta;           // explicit momentum (ignored in Iterate mode)
  const float* atg;     // R*g (Gradient, Step, Iterate, Objective)
  float* out;           // z (Apply), G (Gradient), x_next (Step)
  float invL;           // explicit step (Step mode)
  // Iterate mode: rotation buffers, device state and the group's momentum state
  float* xb[3];
  const IterState* st;
  const GroupMom* gm;
};

// bf16: the BF16-storage variant of the pass (Iterate mode only for pass 3); in Iterate mode a
// variant runs only while the run's storage phase (IterState::bf16) matches it.
int launch_pass1(const GroupDev& g, const StepArgs& a, cudaStream_t s, bool bf16 = false);
int launch_pass2(const GroupDev& g, const IterState* st, cudaStream_t s, bool bf16 = false);
// Pass 3 is two launches: 3a (inverse row transforms into K (*) y) and 3b (prior, gradient,
// update, partial sums); part selects 3a (1), 3b (2) or both (3).
int launch_pass3(const GroupDev& g, const StepArgs& a, Pass3Mode mode, const PriorC& pc, double* partials,
                 int block_offset, cudaStream_t s, bool bf16 = false, int part = 3);
// The passes of n consecutive groups (n <= kMergeMax) of one image side in one launch each, in
// Iterate mode (a.gm is the first group's momentum state).  The groups must share the rows per
// block of passes 1 and 3a and hold their spectra in one chunk (launch_set_ok); pass 3b's blocks
// write the partial-sum rows the groups' separate launches would.
bool launch_set_ok(const GroupDev& first, const GroupDev& g);
int launch_passes_set(const GroupDev* gs, int n, const StepArgs& a, const PriorC& pc, double* partials,
                      int block_offset, cudaStream_t s, bool bf16);
int blocks_pass3(const GroupDev& g);
// slices [c0, c0 + n) of a group as a group of their own (same spectrum buffer)
GroupDev chunk_view(const GroupDev& g, int c0, int n);
// passes 1, 2, 3a of a whole group, chunk by chunk (K (*) y into g.kz, or into the output in
// Apply mode); conv_launches: the kernels that enqueues
int launch_convolution(const GroupDev& g, const StepArgs& a, Pass3Mode mode, const PriorC& pc, cudaStream_t s,
                       bool bf16 = false);
int conv_launches(const GroupDev& g);
// Pass-3b blocks per slice chunk: bands of 4 rows times column blocks of up to 512 columns
// (eight warps of 64 columns).
constexpr int pass3_row_blocks(int N) { return (N / 4) * (N / (64 * (N / 64 < 8 ? N / 64 : 8))); }
// Slices each pass-3 block marches through: enough blocks for about four waves of two
// blocks per SM on 152 SMs, longer marches when the volume has slices to spare.
inline int pass3_slices_per_block(int S, int row_blocks) {
  int chunks = (1216 + row_blocks / 2) / row_blocks;
  if (chunks < 1) chunks = 1;
  if (chunks > S) chunks = S;
  return (S + chunks - 1) / chunks;
}
// slices whose gradient pass 3b computes
inline int pass3_slices(const GroupDev& g) { return g.zn > 0 ? g.zn : g.S; }
// the group's tuned value (tmbir_autotune) or the default rule
inline int pass3_zc(const GroupDev& g, int row_blocks) {
  const int n = pass3_slices(g);
  return g.zc > 0 ? (g.zc < n ? g.zc : n) : pass3_slices_per_block(n, row_blocks);
}
// partial-sum rows pass 3 can write for a group at most (one slice per block)
int max_blocks_pass3(const GroupDev& g);
// cond: the WHILE handle of a device-driven graph loop, set to 0 once the run is done
// (use_cond 1) or also once the run leaves its BF16 phase (use_cond 2); trip_launches:
// kernels of one loop trip, added to IterState::graph_launches.
int launch_finalize(IterState* st, GroupMom* gm, const double* partials, const GroupBlocks& gb, double* log,
                    cudaStream_t s, cudaGraphConditionalHandle cond = 0, int use_cond = 0, int trip_launches = 0);
int launch_sum_partials(const double* partials, int nblocks, double* out, cudaStream_t s);
bool supported_N(int N);
bool block_fft_N(int N);  // sides with a factor 3 or 5 (block-FFT passes, plain twiddle table)
void fft_shape(int N, int* T, int* P);

// setup.cu ------------------------------------------------------------------
int setup_tables(Ctx& c);  // enqueue uploads of twiddles / psi tables into the workspace
int build_kernel_spectrum(Ctx& c, int gi);
// scratch / s: null for the context's setup scratch and stream
// local_out: d_out is the group's own [slice][row][col] buffer (no stacked-image offset)
// weighted: the sinogram rows scaled by the group's per-angle weights (R* W g) when it has them
int backproject(Ctx& c, int gi, const float* d_sino, float* d_out, bool ramp, bool fp64, char* scratch = nullptr,
                cudaStream_t s = nullptr, bool local_out = false, bool weighted = false);
// *d_out = 1/2 sum p[i]^2 (FP64, fixed order; uses the setup scratch); with wts, element i of the
// [slice][angle][bin] rows (na angles, nd bins) counts wts[angle] times
int half_sumsq(Ctx& c, const float* p, size_t n, double* d_out, cudaStream_t s = nullptr, const double* wts = nullptr,
               int na = 0, int nd = 0);
size_t fbp_scratch_bytes(const tmbir_group& g);  // FP32 back-projection scratch of one group
int build_spread_matrix(Ctx& c, int gi);
// R x of one group by the type-2 NUFFT (FP32, Eqs. 3-4) into d_sino (the group's rows of the
// stacked sinogram); uses the setup scratch
int forward_project(Ctx& c, int gi, const float* d_x, float* d_sino, cudaStream_t s = nullptr);
size_t forward_scratch_bytes(const tmbir_group& g);
// d_rx -= d_g over one group's sinogram rows
int residual(Ctx& c, int gi, float* d_rx, const float* d_g, cudaStream_t s = nullptr);
size_t spread_nnz(const tmbir_group& g, int k);
int power_iteration(Ctx& c, int gi, int steps);
int group_gtg(Ctx& c, int gi, const float* d_sino);
void nufft_psi_table(int nmodes, int nfine, int w, double beta, std::vector<double>& out);
size_t setup_scratch_bytes(const tmbir_group& g);

// levels.cu -----------------------------------------------------------------
int launch_upsample_lanczos3(const float* in, int S, int Nc, float* out, cudaStream_t s);
int launch_downsample_sino(const float* in, int S, int na, int nd, int f, float* out, cudaStream_t s);

PriorC make_prior(const tmbir_params& p);
// checks of the prior and optimiser settings shared by the entry points (sets the message)
int check_params(const tmbir_params* p);
// the iteration state of a new run: per group its step constant (from lam_max[i] unless p.L is
// given) and momentum start, 1/2 g.g from gtg[i]; both arrays on the device
int launch_init_state(Ctx& c, const tmbir_params& p, const double* lam_max, const double* gtg, int n_groups,
                      cudaStream_t s);

// argument checks shared by the entry points: a context with a geometry and a bound
// workspace (and, with need_operator, a built operator); sets the error message otherwise
int require_ready(const tmbir_ctx* ctx, bool need_operator);

// static_scratch.cu: looks up the device addresses of the fixed scratch arrays of
// tmbir_normal_apply_static on the current device and caches them.  Looking them up loads
// the module that holds the arrays, which commits their device memory, so tmbir_create calls
// this once for the device current at creation.
int static_scratch_resolve();

}  // namespace tmbir

// the opaque handle of the C ABI
struct tmbir_ctx {
  tmbir::Ctx c;
};
