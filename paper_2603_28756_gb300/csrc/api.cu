// C ABI entry points: context, geometry, workspace layout, and the call sequences of the
// setup, warm-start and iteration phases.  All device work is enqueued on the context stream.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace tmbir {

static thread_local std::string g_last_error;
long long g_launches = 0;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

PriorC make_prior(const tmbir_params& p) {
  PriorC c{};
  c.p = (float)p.p;
  c.q = (float)p.q;
  c.qp = (float)(p.q - p.p);
  c.inv_csig = (float)(1.0 / (p.c * p.sigma));
  c.inv_sig = (float)(1.0 / p.sigma);
  c.inv_sig2 = (float)(1.0 / (p.sigma * p.sigma));
  c.lam = (float)p.lambda;
  const double total = 6.0 + 12.0 / std::sqrt(2.0) + 8.0 / std::sqrt(3.0);
  c.wf = (float)(1.0 / total);
  c.we = (float)(1.0 / std::sqrt(2.0) / total);
  c.wc = (float)(1.0 / std::sqrt(3.0) / total);
  c.q_is_2 = p.q == 2.0 ? 1 : 0;
  c.nonneg = p.nonneg ? 1 : 0;
  c.l2_inv_csig = (float)std::log2(1.0 / (p.c * p.sigma));
  c.qp_l2_inv_csig = (float)((p.q - p.p) * std::log2(1.0 / (p.c * p.sigma)));
  c.l2_inv_sig = (float)std::log2(1.0 / p.sigma);
  return c;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Slices per pass-3 block chosen by tmbir_autotune, by image side and slice count, shared by
// the contexts of this process (0: not tuned).
static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, int> g_tuned_zc;
// slices per spectrum chunk chosen by tmbir_autotune, keyed the same way
static std::map<std::pair<int, int>, int> g_tuned_sc;
// rows per block of passes 1 and 3a (sides with variants), keyed the same way
static std::map<std::pair<int, int>, std::pair<int, int>> g_tuned_rb;

static int tuned_zc(int N, int S) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned_zc.find({N, S});
  return it == g_tuned_zc.end() ? 0 : it->second;
}
static int tuned_sc(int N, int S) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned_sc.find({N, S});
  return it == g_tuned_sc.end() ? 0 : it->second;
}
static std::pair<int, int> tuned_rb(int N, int S) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned_rb.find({N, S});
  return it == g_tuned_rb.end() ? std::make_pair(0, 0) : it->second;
}

// ---------------------------------------------------------------- small device kernels
// lam_max[i], gtg[i]: per-group lambda_max(R*R) and 1/2 g.g gathered into consecutive doubles.
// Every group starts its own momentum sequence with its own step constant.
__global__ void k_init_state(IterState* st, GroupMom* gm, const double* lam_max, const double* gtg, int n_groups,
                             double L_given, double lambda, double sigma, double Fref, double gap_tol, int max_iter,
                             int restart_mode, int bf16, double refine_gap) {
  double gh = 0.0;
  for (int i = 0; i < n_groups; ++i) {
    const double L = L_given > 0.0 ? L_given : 1.01 * lam_max[i] + lambda * 2.0 * (2.0 / (sigma * sigma));
    GroupMom& m = gm[i];
    m.t = 1.0;
    m.beta = 0.0;
    m.L = L;
    m.invL = 1.0 / L;
    m.prev_F = 0.0;
    m.gtg_half = gtg[i];
    m.restarts = 0;
    m.pad = 0;
    gh += gtg[i];
  }
  st->t = 1.0;
  st->beta = 0.0;
  st->L = gm[0].L;
  st->invL = gm[0].invL;
  st->lambda = lambda;
  st->gtg_half = gh;
  st->F0 = gh;
  st->Fref = Fref;
  st->gap_tol = gap_tol;
  st->last_F = st->last_gap = st->last_gg = st->last_dot = 0.0;
  st->k = 0;
  st->max_iter = max_iter;
  st->restarts = 0;
  st->cur = 0;
  st->done = max_iter <= 0 ? 1 : 0;
  st->status = 0;
  st->restart_mode = restart_mode;
  st->log_cap = kLogCap;
  st->prev_F = 0.0;
  st->bf16 = bf16;
  st->refine_gap = refine_gap;
}

// End of a run: bring the rotation to its start position, x_k in slot 0 (the caller's buffer)
// and x_{k-1} in slot 2, so the state can be exported or resumed (k_rotation_reset then sets
// the rotation index to 0).
__global__ void k_gather_final(const IterState* st, float* x0, float* x1, float* x2, size_t n) {
  const int cur = st->cur;
  if (cur == 0) return;
  float4* a = reinterpret_cast<float4*>(x0);
  float4* b = reinterpret_cast<float4*>(x1);
  float4* c = reinterpret_cast<float4*>(x2);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n / 4; i += (size_t)gridDim.x * blockDim.x) {
    if (cur == 1) {  // x_k in slot 1, x_{k-1} in slot 0
      const float4 xk = b[i], xp = a[i];
      a[i] = xk;
      c[i] = xp;
    } else {  // x_k in slot 2, x_{k-1} in slot 1
      const float4 xk = c[i], xp = b[i];
      a[i] = xk;
      c[i] = xp;
    }
  }
}
__global__ void k_rotation_reset(IterState* st) { st->cur = 0; }

int launch_init_state(Ctx& c, const tmbir_params& p, const double* lam_max, const double* gtg, int n_groups,
                      cudaStream_t s) {
  const bool bf16 = p.spectra == TMBIR_SPECTRA_BF16;
  k_init_state<<<1, 1, 0, s>>>(c.state, c.gmom, lam_max, gtg, n_groups, p.L, p.lambda, p.sigma, p.F_ref, p.gap_tol,
                               p.max_iter, p.restart, bf16 ? 1 : 0, p.refine_gap);
  TMBIR_CHECK_LAUNCH();
  return TMBIR_OK;
}

// continue a run from the current state: max_iter more iterations with new stop settings
__global__ void k_resume_state(IterState* st, double Fref, double gap_tol, int max_iter, int restart_mode, int bf16,
                               double refine_gap) {
  st->max_iter = st->k + max_iter;
  st->Fref = Fref;
  st->gap_tol = gap_tol;
  st->restart_mode = restart_mode;
  st->bf16 = bf16;
  st->refine_gap = refine_gap;
  st->done = max_iter <= 0 ? 1 : 0;
  st->status = 0;
}

__global__ void k_scale_copy(const float* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) out[i] = in[i];
}

}  // namespace tmbir

using namespace tmbir;

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

#define REQUIRE(cond, code, msg) \
  do {                           \
    if (!(cond)) return set_error(code, msg); \
  } while (0)

int tmbir::require_ready(const tmbir_ctx* ctx, bool need_operator) {
  if (!ctx) return set_error(TMBIR_ERR_ARG, "ctx is NULL");
  if (ctx->c.groups.empty()) return set_error(TMBIR_ERR_STATE, "no geometry set");
  if (!ctx->c.ws) return set_error(TMBIR_ERR_WORKSPACE, "no workspace bound");
  if (need_operator && !ctx->c.operator_built) return set_error(TMBIR_ERR_STATE, "operator not built");
  return TMBIR_OK;
}

int tmbir::check_params(const tmbir_params* p) {
  if (!p) return set_error(TMBIR_ERR_ARG, "params is NULL");
  if (!(p->p >= 1.0 && p->q >= p->p && p->q <= 4.0)) return set_error(TMBIR_ERR_ARG, "need 1 <= p <= q <= 4");
  if (!(p->c > 0.0 && p->sigma > 0.0 && p->lambda >= 0.0)) return set_error(TMBIR_ERR_ARG, "need c > 0, sigma > 0, lambda >= 0");
  if (p->L <= 0.0 && p->q != 2.0) return set_error(TMBIR_ERR_ARG, "automatic L needs q = 2; pass L > 0");
  if (p->restart != TMBIR_RESTART_GRADIENT && p->restart != TMBIR_RESTART_NONE && p->restart != TMBIR_RESTART_FUNCTION)
    return set_error(TMBIR_ERR_ARG, "unknown restart mode");
  if ((p->spectra != TMBIR_SPECTRA_FP32 && p->spectra != TMBIR_SPECTRA_BF16) || !(p->refine_gap >= 0.0))
    return set_error(TMBIR_ERR_ARG, "spectra must be FP32 or BF16 and refine_gap >= 0");
  return TMBIR_OK;
}

extern "C" {

const char* tmbir_last_error(void) { return g_last_error.c_str(); }

int tmbir_create(tmbir_ctx** out, void* stream) {
  REQUIRE(out != nullptr, TMBIR_ERR_ARG, "tmbir_create: out is NULL");
  int dev_count = 0;
  cudaError_t e = cudaGetDeviceCount(&dev_count);
  if (e != cudaSuccess || dev_count == 0) return set_error(TMBIR_ERR_CUDA, "tmbir_create: no CUDA device");
  // commit the fixed scratch arrays of tmbir_normal_apply_static on this device now, not at
  // that entry point's first call (and refresh their cached addresses, e.g. after a reset)
  if (int rc = static_scratch_resolve()) return rc;
  tmbir_ctx* ctx = new tmbir_ctx();
  ctx->c.stream = (cudaStream_t)stream;
  *out = ctx;
  g_last_error.clear();
  return TMBIR_OK;
}

int tmbir_destroy(tmbir_ctx* ctx) {
  if (!ctx) return TMBIR_OK;
  if (ctx->c.graph_exec) cudaGraphExecDestroy(ctx->c.graph_exec);
  if (ctx->c.ev_fork) cudaEventDestroy(ctx->c.ev_fork);
  if (ctx->c.ev_join) cudaEventDestroy(ctx->c.ev_join);
  if (ctx->c.aux) cudaStreamDestroy(ctx->c.aux);
  for (int s = 0; s < 2; ++s) {
    if (ctx->c.ev_in[s]) cudaEventDestroy(ctx->c.ev_in[s]);
    if (ctx->c.ev_comp[s]) cudaEventDestroy(ctx->c.ev_comp[s]);
    if (ctx->c.ev_out[s]) cudaEventDestroy(ctx->c.ev_out[s]);
  }
  if (ctx->c.ev_start) cudaEventDestroy(ctx->c.ev_start);
  if (ctx->c.s_in) cudaStreamDestroy(ctx->c.s_in);
  if (ctx->c.s_out) cudaStreamDestroy(ctx->c.s_out);
  delete ctx;
  return TMBIR_OK;
}

int tmbir_set_geometry(tmbir_ctx* ctx, int n_groups, const tmbir_group* groups) {
  TMBIR_TRACE("tmbir_set_geometry");
  REQUIRE(ctx != nullptr, TMBIR_ERR_ARG, "set_geometry: ctx is NULL");
  REQUIRE(n_groups >= 1 && groups != nullptr, TMBIR_ERR_ARG, "set_geometry: need at least one group");
  REQUIRE(n_groups <= kMaxGroups, TMBIR_ERR_ARG, "set_geometry: at most 64 groups");
  Ctx& c = ctx->c;
  std::vector<tmbir_group> gs(groups, groups + n_groups);
  std::vector<std::vector<double>> angs(n_groups);
  for (int i = 0; i < n_groups; ++i) {
    const tmbir_group& g = gs[i];
    REQUIRE(supported_N(g.N), TMBIR_ERR_SHAPE, "set_geometry: N must be a power of two in [64, 2048], or 1536 or 2560");
    REQUIRE(g.n_det == g.N, TMBIR_ERR_SHAPE, "set_geometry: n_det must equal N");
    REQUIRE(g.n_angles >= 1 && g.n_angles <= 1 << 16, TMBIR_ERR_ARG, "set_geometry: n_angles out of range");
    REQUIRE(g.angles != nullptr, TMBIR_ERR_ARG, "set_geometry: angles is NULL");
    REQUIRE(g.n_slices >= 1, TMBIR_ERR_ARG, "set_geometry: n_slices must be >= 1");
    REQUIRE(g.span > 0.0 && std::isfinite(g.span), TMBIR_ERR_ARG, "set_geometry: span must be positive");
    angs[i].assign(g.angles, g.angles + g.n_angles);
    for (double a : angs[i]) REQUIRE(std::isfinite(a), TMBIR_ERR_ARG, "set_geometry: non-finite angle");
    gs[i].angles = nullptr;
  }
  if (c.graph_exec) {
    cudaGraphExecDestroy(c.graph_exec);
    c.graph_exec = nullptr;
  }
  c.groups = gs;
  c.angles = angs;
  c.gdev.assign(n_groups, GroupDev{});
  c.ws = nullptr;
  c.ws_bytes = 0;
  c.operator_built = false;
  c.nufft_beta64 = 2.30 * 12;
  c.psiK_h.assign(n_groups, {});
  for (int k = 0; k < 2; ++k) c.psiS_h[k].assign(n_groups, {});
  c.geom_ready.assign(n_groups, false);
  c.spread_ready.assign(n_groups, false);
  c.weights.assign(n_groups, {});

  // workspace layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align_up(off, 256);
    size_t o = off;
    off += bytes;
    return o;
  };
  c.off_state = take(sizeof(IterState));
  c.off_gmom = take((size_t)n_groups * sizeof(GroupMom));
  c.off_dscal = take((16 + 2 * (size_t)n_groups) * sizeof(double));
  int max_blocks = 0, slices = 0;
  size_t voxels = 0, sino = 0, scratch = 0, fbp_scratch = 0;
  for (int i = 0; i < n_groups; ++i) {
    GroupDev tmp{};
    tmp.N = gs[i].N;
    tmp.S = gs[i].n_slices;
    max_blocks += max_blocks_pass3(tmp);  // any slices-per-block choice fits
    voxels += (size_t)gs[i].n_slices * gs[i].N * gs[i].N;
    sino += (size_t)gs[i].n_slices * gs[i].n_angles * gs[i].n_det;
    scratch = std::max(scratch, setup_scratch_bytes(gs[i]));
    fbp_scratch = std::max(fbp_scratch, fbp_scratch_bytes(gs[i]));
  }
  c.max_blocks = std::max(max_blocks, 1);
  c.off_partials = take((size_t)c.max_blocks * kParts * sizeof(double));
  c.off_log = take((size_t)kLogCap * 4 * sizeof(double));
  c.off_chat.resize(n_groups);
  c.off_twN.resize(n_groups);
  c.off_twM.resize(n_groups);
  c.off_spec.resize(n_groups);
  c.off_kz.resize(n_groups);
  c.off_ang.resize(n_groups);
  c.off_K.resize(n_groups);
  c.off_psiK.resize(n_groups);
  for (int k = 0; k < 2; ++k) {
    c.off_sp_psi[k].resize(n_groups);
    c.off_sp_ptr[k].resize(n_groups);
    c.off_sp_idx[k].resize(n_groups);
    c.off_sp_wt[k].resize(n_groups);
  }
  c.off_lam.resize(n_groups);
  c.off_gtg.resize(n_groups);
  c.off_wts.resize(n_groups);
  for (int i = 0; i < n_groups; ++i) {
    const size_t N = gs[i].N;
    c.off_chat[i] = take((N + 1) * 2 * N * sizeof(float));
    c.off_twN[i] = take(N * sizeof(float2));
    c.off_twM[i] = take(N * sizeof(float2));
    c.off_spec[i] = take((size_t)gs[i].n_slices * (N + 1) * N * sizeof(float2));
    c.off_kz[i] = take((size_t)gs[i].n_slices * N * N * sizeof(float));
    c.off_ang[i] = take(gs[i].n_angles * sizeof(double));
    c.off_K[i] = take((2 * N - 1) * (2 * N - 1) * sizeof(double));
    c.off_psiK[i] = take((2 * N - 1) * sizeof(double));
    for (int k = 0; k < 2; ++k) {
      const size_t nf = spread_grid(k, (int)N);
      c.off_sp_psi[k][i] = take(N * sizeof(double));
      c.off_sp_ptr[k][i] = take((nf * nf + 1) * sizeof(int));
      c.off_sp_idx[k][i] = take(spread_nnz(gs[i], k) * sizeof(int));
      c.off_sp_wt[k][i] = take(spread_nnz(gs[i], k) * sizeof(double));
    }
    c.off_lam[i] = take(sizeof(double));
    c.off_gtg[i] = take(sizeof(double));
    c.off_wts[i] = take(gs[i].n_angles * sizeof(double));
    nufft_psi_table(2 * N - 1, 4 * N, 12, c.nufft_beta64, c.psiK_h[i]);
    for (int k = 0; k < 2; ++k)
      nufft_psi_table(N, spread_grid(k, (int)N), kSpreadWidth[k], spread_beta(k), c.psiS_h[k][i]);
  }
  c.off_xbuf0 = take(voxels * sizeof(float));
  c.off_xbuf1 = take(voxels * sizeof(float));
  c.off_scratch = take(scratch);
  c.off_fbp_scratch = take(fbp_scratch);
  c.off_sino_tmp = take(sino * sizeof(float));
  c.scratch_bytes = scratch;
  c.ws_need = align_up(off, 256);
  c.total_voxels = voxels;
  c.total_sino = sino;
  c.total_slices = slices;
  int s0 = 0;
  size_t io = 0, so = 0;
  for (int i = 0; i < n_groups; ++i) {
    c.gdev[i].slice0 = s0;
    c.gdev[i].img_off = io;
    c.gdev[i].sino_off = so;
    s0 += gs[i].n_slices;
    io += (size_t)gs[i].n_slices * gs[i].N * gs[i].N;
    so += (size_t)gs[i].n_slices * gs[i].n_angles * gs[i].n_det;
  }
  c.total_slices = s0;
  g_last_error.clear();
  return TMBIR_OK;
}

int tmbir_workspace_size(const tmbir_ctx* ctx, size_t* bytes) {
  REQUIRE(ctx != nullptr && bytes != nullptr, TMBIR_ERR_ARG, "workspace_size: NULL argument");
  REQUIRE(!ctx->c.groups.empty(), TMBIR_ERR_STATE, "workspace_size: no geometry");
  *bytes = ctx->c.ws_need;
  return TMBIR_OK;
}

int tmbir_set_workspace(tmbir_ctx* ctx, void* d_ws, size_t bytes) {
  TMBIR_TRACE("tmbir_set_workspace");
  REQUIRE(ctx != nullptr, TMBIR_ERR_ARG, "set_workspace: ctx is NULL");
  Ctx& c = ctx->c;
  REQUIRE(!c.groups.empty(), TMBIR_ERR_STATE, "set_workspace: no geometry");
  REQUIRE(d_ws != nullptr, TMBIR_ERR_ARG, "set_workspace: workspace is NULL");
  REQUIRE(((uintptr_t)d_ws & 255u) == 0, TMBIR_ERR_ARG, "set_workspace: workspace must be 256-byte aligned");
  REQUIRE(bytes >= c.ws_need, TMBIR_ERR_WORKSPACE, "set_workspace: workspace too small");
  if (c.graph_exec) {
    cudaGraphExecDestroy(c.graph_exec);
    c.graph_exec = nullptr;
  }
  char* ws = static_cast<char*>(d_ws);
  c.ws = ws;
  c.ws_bytes = bytes;
  c.state = reinterpret_cast<IterState*>(ws + c.off_state);
  c.gmom = reinterpret_cast<GroupMom*>(ws + c.off_gmom);
  c.dscal = reinterpret_cast<double*>(ws + c.off_dscal);
  c.partials = reinterpret_cast<double*>(ws + c.off_partials);
  c.log = reinterpret_cast<double*>(ws + c.off_log);
  c.xbuf[0] = reinterpret_cast<float*>(ws + c.off_xbuf0);
  c.xbuf[1] = reinterpret_cast<float*>(ws + c.off_xbuf1);
  c.scratch = ws + c.off_scratch;
  c.fbp_scratch = ws + c.off_fbp_scratch;
  c.sino_tmp = reinterpret_cast<float*>(ws + c.off_sino_tmp);
  TMBIR_CUDA(cudaMemsetAsync(c.state, 0, sizeof(IterState), c.stream));
  TMBIR_CUDA(cudaMemsetAsync(c.gmom, 0, c.groups.size() * sizeof(GroupMom), c.stream));
  c.state_ready = false;
  for (size_t i = 0; i < c.groups.size(); ++i) {
    const tmbir_group& g = c.groups[i];
    GroupDev& d = c.gdev[i];
    d.N = g.N;
    d.nd = g.n_det;
    d.na = g.n_angles;
    d.S = g.n_slices;
    d.span = (float)g.span;
    d.zc = tuned_zc(d.N, d.S);
    d.sc = tuned_sc(d.N, d.S);
    d.rb1 = tuned_rb(d.N, d.S).first;
    d.rb3 = tuned_rb(d.N, d.S).second;
    d.chat = reinterpret_cast<float*>(ws + c.off_chat[i]);
    d.twN = reinterpret_cast<float2*>(ws + c.off_twN[i]);
    d.twM = reinterpret_cast<float2*>(ws + c.off_twM[i]);
    d.spec = reinterpret_cast<float2*>(ws + c.off_spec[i]);
    d.kz = reinterpret_cast<float*>(ws + c.off_kz[i]);
    d.angles = reinterpret_cast<double*>(ws + c.off_ang[i]);
    d.K = reinterpret_cast<double*>(ws + c.off_K[i]);
    d.psiK = reinterpret_cast<double*>(ws + c.off_psiK[i]);
    for (int k = 0; k < 2; ++k) {
      d.sp[k].nf = spread_grid(k, g.N);
      d.sp[k].psi = reinterpret_cast<double*>(ws + c.off_sp_psi[k][i]);
      d.sp[k].ptr = reinterpret_cast<int*>(ws + c.off_sp_ptr[k][i]);
      d.sp[k].idx = reinterpret_cast<int*>(ws + c.off_sp_idx[k][i]);
      d.sp[k].wt = reinterpret_cast<double*>(ws + c.off_sp_wt[k][i]);
    }
    d.lam_max = reinterpret_cast<double*>(ws + c.off_lam[i]);
    d.gtg = reinterpret_cast<double*>(ws + c.off_gtg[i]);
    d.wts = nullptr;
    if (!c.weights[i].empty()) {
      double* w = reinterpret_cast<double*>(ws + c.off_wts[i]);
      TMBIR_CUDA(cudaMemcpyAsync(w, c.weights[i].data(), c.weights[i].size() * sizeof(double), cudaMemcpyHostToDevice,
                                 c.stream));
      d.wts = w;
    }
    // twiddle tables: twN[k][t] = exp(-2 pi i t k / N) in the group-FFT layout (the plain
    // table exp(-2 pi i j / N) for the block-FFT sides), twM[n] = exp(-2 pi i n / 2N)
    int T, P;
    fft_shape(g.N, &T, &P);
    std::vector<float2> twN((size_t)T * P), twM(g.N);
    for (int k = 0; k < P; ++k)
      for (int t = 0; t < T; ++t) {
        const long long q = block_fft_N(g.N) ? (long long)k * T + t : (long long)t * k % g.N;
        const double a = -2.0 * M_PI * (double)q / g.N;
        twN[(size_t)k * T + t] = make_float2((float)std::cos(a), (float)std::sin(a));
      }
    for (int n = 0; n < g.N; ++n) {
      const double a = -M_PI * (double)n / g.N;
      twM[n] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    TMBIR_CUDA(cudaMemcpyAsync(d.twN, twN.data(), twN.size() * sizeof(float2), cudaMemcpyHostToDevice, c.stream));
    TMBIR_CUDA(cudaMemcpyAsync(d.twM, twM.data(), twM.size() * sizeof(float2), cudaMemcpyHostToDevice, c.stream));
    TMBIR_CUDA(cudaMemcpyAsync(d.angles, c.angles[i].data(), c.angles[i].size() * sizeof(double), cudaMemcpyHostToDevice,
                               c.stream));
    TMBIR_CUDA(cudaMemcpyAsync(d.psiK, c.psiK_h[i].data(), c.psiK_h[i].size() * sizeof(double), cudaMemcpyHostToDevice,
                               c.stream));
    for (int k = 0; k < 2; ++k)
      TMBIR_CUDA(cudaMemcpyAsync(d.sp[k].psi, c.psiS_h[k][i].data(), c.psiS_h[k][i].size() * sizeof(double),
                                 cudaMemcpyHostToDevice, c.stream));

  }
  // pageable host sources: make sure the copies have consumed them before the vectors go away
  TMBIR_CUDA(cudaStreamSynchronize(c.stream));
  c.operator_built = false;
  c.geom_ready.assign(c.groups.size(), false);
  c.spread_ready.assign(c.groups.size(), false);
  return TMBIR_OK;
}


int tmbir_set_angle_weights(tmbir_ctx* ctx, int group, const double* h_w) {
  TMBIR_TRACE("tmbir_set_angle_weights");
  REQUIRE(ctx != nullptr, TMBIR_ERR_ARG, "set_angle_weights: ctx is NULL");
  Ctx& c = ctx->c;
  REQUIRE(!c.groups.empty(), TMBIR_ERR_STATE, "set_angle_weights: no geometry");
  REQUIRE(group >= 0 && group < (int)c.groups.size(), TMBIR_ERR_ARG, "set_angle_weights: no such group");
  const int na = c.groups[group].n_angles;
  std::vector<double> w;
  if (h_w) {
    w.assign(h_w, h_w + na);
    for (double v : w)
      REQUIRE(std::isfinite(v) && v >= 0.0 && v <= 1.0, TMBIR_ERR_ARG, "set_angle_weights: weights must lie in [0, 1]");
  }
  c.weights[group] = w;
  GroupDev& d = c.gdev[group];
  d.wts = nullptr;
  if (c.ws && !w.empty()) {
    double* dw = reinterpret_cast<double*>(c.ws + c.off_wts[group]);
    TMBIR_CUDA(cudaMemcpyAsync(dw, c.weights[group].data(), na * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    TMBIR_CUDA(cudaStreamSynchronize(c.stream));
    d.wts = dw;
  }
  // K, lambda_max, R*g and 1/2 g.g depend on the weights: rebuilt by the next build call
  c.geom_ready[group] = false;
  c.operator_built = false;
  c.state_ready = false;
  if (c.graph_exec) {
    cudaGraphExecDestroy(c.graph_exec);
    c.graph_exec = nullptr;
  }
  return TMBIR_OK;
}

int tmbir_build_operator(tmbir_ctx* ctx, const float* d_sino, float* d_atg) {
  TMBIR_TRACE("tmbir_build_operator");
  if (int e = require_ready(ctx, false)) return e;
  REQUIRE(d_sino && d_atg && aligned16(d_sino) && aligned16(d_atg), TMBIR_ERR_ARG,
          "build_operator: sinogram and output must be non-NULL and 16-byte aligned");
  Ctx& c = ctx->c;
  for (size_t i = 0; i < c.groups.size(); ++i) {
    // geometry-only parts: once per geometry and workspace binding
    if (!c.spread_ready[i]) {
      if (int e = build_spread_matrix(c, (int)i)) return e;
      c.spread_ready[i] = true;
    }
    if (!c.geom_ready[i]) {
      if (int e = build_kernel_spectrum(c, (int)i)) return e;
      if (int e = power_iteration(c, (int)i, 100)) return e;
      c.geom_ready[i] = true;
    }
    // data parts: every call
    if (int e = backproject(c, (int)i, d_sino, d_atg, false, true, nullptr, nullptr, false, true)) return e;
    if (int e = group_gtg(c, (int)i, d_sino)) return e;
  }
  c.operator_built = true;
  return TMBIR_OK;
}

int tmbir_build_operator_fp32(tmbir_ctx* ctx, const float* d_sino, float* d_atg) {
  TMBIR_TRACE("tmbir_build_operator_fp32");
  if (int e = require_ready(ctx, false)) return e;
  REQUIRE(d_sino && d_atg && aligned16(d_sino) && aligned16(d_atg), TMBIR_ERR_ARG,
          "build_operator_fp32: sinogram and output must be non-NULL and 16-byte aligned");
  Ctx& c = ctx->c;
  for (size_t i = 0; i < c.groups.size(); ++i) {
    if (!c.spread_ready[i]) {
      if (int e = build_spread_matrix(c, (int)i)) return e;
      c.spread_ready[i] = true;
    }
    if (!c.geom_ready[i]) {
      if (int e = build_kernel_spectrum(c, (int)i)) return e;
      if (int e = power_iteration(c, (int)i, 100)) return e;
      c.geom_ready[i] = true;
    }
    // R*g by the FP32 back-projection (the FBP start's transform, without the ramp filter)
    if (int e = backproject(c, (int)i, d_sino, d_atg, false, false, nullptr, nullptr, false, true)) return e;
    if (int e = group_gtg(c, (int)i, d_sino)) return e;
  }
  c.operator_built = true;
  return TMBIR_OK;
}

// build_operator and fbp in one call: R*g (FP64) on the context stream while the FBP start
// (FP32, its own scratch) runs on a second stream, joined before the call returns its work.
int tmbir_build_operator_fbp(tmbir_ctx* ctx, const float* d_sino, float* d_atg, float* d_x0) {
  TMBIR_TRACE("tmbir_build_operator_fbp");
  if (int e = require_ready(ctx, false)) return e;
  REQUIRE(d_sino && d_atg && d_x0 && aligned16(d_sino) && aligned16(d_atg) && aligned16(d_x0), TMBIR_ERR_ARG,
          "build_operator_fbp: buffers must be non-NULL and 16-byte aligned");
  REQUIRE(d_atg != d_x0, TMBIR_ERR_ARG, "build_operator_fbp: R*g and the start must be different buffers");
  Ctx& c = ctx->c;
  REQUIRE(c.stream != nullptr, TMBIR_ERR_ARG, "build_operator_fbp: needs a context stream (not the legacy stream)");
  if (!c.aux) {
    TMBIR_CUDA(cudaStreamCreateWithFlags(&c.aux, cudaStreamNonBlocking));
    TMBIR_CUDA(cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
    TMBIR_CUDA(cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming));
  }
  for (size_t i = 0; i < c.groups.size(); ++i) {
    // geometry-only parts first: both branches read the spreading matrix
    if (!c.spread_ready[i]) {
      if (int e = build_spread_matrix(c, (int)i)) return e;
      c.spread_ready[i] = true;
    }
    if (!c.geom_ready[i]) {
      if (int e = build_kernel_spectrum(c, (int)i)) return e;
      if (int e = power_iteration(c, (int)i, 100)) return e;
      c.geom_ready[i] = true;
    }
  }
  TMBIR_CUDA(cudaEventRecord(c.ev_fork, c.stream));
  TMBIR_CUDA(cudaStreamWaitEvent(c.aux, c.ev_fork, 0));
  int rc = TMBIR_OK;
  for (size_t i = 0; i < c.groups.size() && rc == TMBIR_OK; ++i)
    rc = backproject(c, (int)i, d_sino, d_x0, true, false, c.fbp_scratch, c.aux);
  for (size_t i = 0; i < c.groups.size() && rc == TMBIR_OK; ++i) {
    if ((rc = backproject(c, (int)i, d_sino, d_atg, false, true, nullptr, nullptr, false, true))) break;
    rc = group_gtg(c, (int)i, d_sino);
  }
  // join whatever was enqueued, also after an error
  cudaError_t e1 = cudaEventRecord(c.ev_join, c.aux);
  cudaError_t e2 = cudaStreamWaitEvent(c.stream, c.ev_join, 0);
  if (rc) return rc;
  if (e1 != cudaSuccess || e2 != cudaSuccess) return set_error(TMBIR_ERR_CUDA, "build_operator_fbp: stream join failed");
  c.operator_built = true;
  return TMBIR_OK;
}

int tmbir_fbp(tmbir_ctx* ctx, const float* d_sino, float* d_x0) {
  TMBIR_TRACE("tmbir_fbp");
  if (int e = require_ready(ctx, false)) return e;
  REQUIRE(d_sino && d_x0 && aligned16(d_sino) && aligned16(d_x0), TMBIR_ERR_ARG,
          "fbp: sinogram and output must be non-NULL and 16-byte aligned");
  Ctx& c = ctx->c;
  for (size_t i = 0; i < c.groups.size(); ++i) {
    if (!c.spread_ready[i]) {
      if (int e = build_spread_matrix(c, (int)i)) return e;
      c.spread_ready[i] = true;
    }
    if (int e = backproject(c, (int)i, d_sino, d_x0, true, false)) return e;
  }
  return TMBIR_OK;
}

// first partial-sum row of each group's pass-3b blocks
static GroupBlocks group_blocks(const Ctx& c) {
  GroupBlocks gb{};
  gb.n = (int)c.gdev.size();
  for (int i = 0; i < gb.n; ++i) gb.off[i + 1] = gb.off[i] + blocks_pass3(c.gdev[i]);
  return gb;
}

// The launch sets of an iteration: runs of consecutive groups (at most kMergeMax) that one launch
// per pass covers, [first, end) each; a group that cannot share launches forms a run of its own.
static std::vector<std::pair<int, int>> launch_runs(const Ctx& c) {
  std::vector<std::pair<int, int>> runs;
  const int ng = (int)c.gdev.size();
  for (int i = 0; i < ng;) {
    int j = i + 1;
    while (j < ng && j - i < kMergeMax && launch_set_ok(c.gdev[i], c.gdev[j])) ++j;
    runs.emplace_back(i, j);
    i = j;
  }
  return runs;
}
static int run_launches(const Ctx& c, const std::pair<int, int>& r) {
  return r.second - r.first > 1 ? 4 : conv_launches(c.gdev[r.first]) + 1;
}

// Passes 1-3 of every group in Iterate mode, FP32 or BF16 storage variant: one launch per pass
// for each run of groups that can share launches (consecutive groups of one image side, e.g.
// the angle counts of one side in an uneven batch).  *nblocks receives the number of
// partial-sum rows they write (each group's rows where its own launches would put them).
static int enqueue_passes(Ctx& c, float* d_x, const float* d_atg, const PriorC& pc, bool bf16, int* nblocks) {
  StepArgs a{};
  a.atg = d_atg;
  a.xb[0] = d_x;
  a.xb[1] = c.xbuf[0];
  a.xb[2] = c.xbuf[1];
  a.st = c.state;
  int off = 0;
  for (const auto& r : launch_runs(c)) {
    a.gm = c.gmom + r.first;
    if (r.second - r.first > 1) {
      if (int e = launch_passes_set(c.gdev.data() + r.first, r.second - r.first, a, pc, c.partials, off, c.stream,
                                    bf16))
        return e;
    } else {
      const GroupDev& g = c.gdev[r.first];
      if (int e = launch_convolution(g, a, Pass3Mode::Iterate, pc, c.stream, bf16)) return e;
      if (int e = launch_pass3(g, a, Pass3Mode::Iterate, pc, c.partials, off, c.stream, bf16, 2)) return e;
    }
    for (int i = r.first; i < r.second; ++i) off += blocks_pass3(c.gdev[i]);
  }
  *nblocks = off;
  return TMBIR_OK;
}

// iters eager iterations.  kind (see Ctx::graph_kind) selects the storage variants: every
// variant checks the run's phase on the device, so a BF16 run with refinement enqueues both
// and the one that does not match leaves at once.
static int enqueue_iterations(Ctx& c, float* d_x, const float* d_atg, const PriorC& pc, int iters, int kind) {
  for (int k = 0; k < iters; ++k) {
    int nb = 0;
    if (kind >= 2)
      if (int e = enqueue_passes(c, d_x, d_atg, pc, true, &nb)) return e;
    if (kind != 2)
      if (int e = enqueue_passes(c, d_x, d_atg, pc, false, &nb)) return e;
    if (int e = launch_finalize(c.state, c.gmom, c.partials, group_blocks(c), c.log, c.stream)) return e;
  }
  return TMBIR_OK;
}

// one trip of a device-driven loop: the passes of one storage variant and the finalize kernel
static int enqueue_trip(Ctx& c, float* d_x, const float* d_atg, const PriorC& pc, bool bf16,
                        cudaGraphConditionalHandle cond, int use_cond) {
  int nb = 0;
  if (int e = enqueue_passes(c, d_x, d_atg, pc, bf16, &nb)) return e;
  int trip_launches = 1;
  for (const auto& r : launch_runs(c)) trip_launches += run_launches(c, r);
  return launch_finalize(c.state, c.gmom, c.partials, group_blocks(c), c.log, c.stream, cond, use_cond, trip_launches);
}

// Appends a WHILE node after `dep` (may be null) whose body is one trip; *node receives it.
static int add_loop(Ctx& c, cudaGraph_t gr, cudaGraphNode_t* dep, float* d_x, const float* d_atg, const PriorC& pc,
                    bool bf16, int use_cond, cudaGraphNode_t* node) {
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, gr, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return set_error(TMBIR_ERR_CUDA, "graph: conditional handle");
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  if (cudaGraphAddNode(node, gr, dep, nullptr, dep ? 1 : 0, &np) != cudaSuccess)
    return set_error(TMBIR_ERR_CUDA, "graph: conditional node");
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(c.stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess)
    return set_error(TMBIR_ERR_CUDA, "graph: begin capture");
  const long long n0 = __atomic_load_n(&g_launches, __ATOMIC_RELAXED);
  int e = enqueue_trip(c, d_x, d_atg, pc, bf16, h, use_cond);
  cudaGraph_t captured = nullptr;
  cudaError_t ce = cudaStreamEndCapture(c.stream, &captured);
  // captured launches run on replay, where the finalize kernel counts them on the device
  __atomic_sub_fetch(&g_launches, __atomic_load_n(&g_launches, __ATOMIC_RELAXED) - n0, __ATOMIC_RELAXED);
  if (e) return e;
  if (ce != cudaSuccess) return set_error(TMBIR_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  return TMBIR_OK;
}

// One executable graph of WHILE nodes, each repeating one iteration until its finalize kernel
// clears the condition: kind 1 a FP32 loop; kind 2 a BF16 loop; kind 3 a BF16 loop that ends
// at the refinement switch followed by a FP32 loop.
static int build_loop_graph(Ctx& c, float* d_x, const float* d_atg, const PriorC& pc, int kind) {
  cudaGraph_t gr = nullptr;
  TMBIR_CUDA(cudaGraphCreate(&gr, 0));
  cudaGraphNode_t first = nullptr, second = nullptr;
  int e = TMBIR_OK;
  if (kind >= 2) e = add_loop(c, gr, nullptr, d_x, d_atg, pc, true, kind == 3 ? 2 : 1, &first);
  if (!e && kind != 2) e = add_loop(c, gr, first ? &first : nullptr, d_x, d_atg, pc, false, 1, &second);
  if (!e && cudaGraphInstantiate(&c.graph_exec, gr, 0) != cudaSuccess) {
    c.graph_exec = nullptr;
    e = set_error(TMBIR_ERR_CUDA, "graph: instantiate");
  }
  cudaGraphDestroy(gr);
  return e;
}

int tmbir_reconstruct(tmbir_ctx* ctx, float* d_x, const float* d_atg, const tmbir_params* prm, tmbir_stats* h_stats) {
  TMBIR_TRACE("tmbir_reconstruct");
  if (int e = require_ready(ctx, true)) return e;
  if (int e = check_params(prm)) return e;
  REQUIRE(d_x && d_atg && aligned16(d_x) && aligned16(d_atg), TMBIR_ERR_ARG,
          "reconstruct: image and R*g must be non-NULL and 16-byte aligned");
  REQUIRE(prm->max_iter >= 0 && prm->max_iter <= kLogCap, TMBIR_ERR_ARG, "reconstruct: max_iter out of range");
  Ctx& c = ctx->c;
  cudaStream_t s = c.stream;
  const PriorC pc = make_prior(*prm);
  // gather the per-group lambda_max and 1/2 g.g into dscal[16 .. 16 + 2 ng)
  const int ng = (int)c.gdev.size();
  for (int i = 0; i < ng; ++i) {
    TMBIR_CUDA(cudaMemcpyAsync(c.dscal + 16 + i, c.gdev[i].lam_max, sizeof(double), cudaMemcpyDeviceToDevice, s));
    TMBIR_CUDA(cudaMemcpyAsync(c.dscal + 16 + ng + i, c.gdev[i].gtg, sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  const bool bf16 = prm->spectra == TMBIR_SPECTRA_BF16;
  if (prm->resume) {
    // continue the previous (or imported) run: x_k is d_x, x_{k-1} is in slot 2
    REQUIRE(c.state_ready, TMBIR_ERR_STATE, "reconstruct: nothing to resume (no run or imported state)");
    k_resume_state<<<1, 1, 0, s>>>(c.state, prm->F_ref, prm->gap_tol, prm->max_iter, prm->restart, bf16 ? 1 : 0,
                                   prm->refine_gap);
    TMBIR_CHECK_LAUNCH();
  } else {
    k_init_state<<<1, 1, 0, s>>>(c.state, c.gmom, c.dscal + 16, c.dscal + 16 + ng, ng, prm->L, prm->lambda,
                                 prm->sigma, prm->F_ref, prm->gap_tol, prm->max_iter, prm->restart, bf16 ? 1 : 0,
                                 prm->refine_gap);
    TMBIR_CHECK_LAUNCH();
    // x_{-1} = x_0 so that the first (beta = 0) extrapolation reads finite values
    TMBIR_CUDA(cudaMemcpyAsync(c.xbuf[1], d_x, c.total_voxels * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  const int iters = prm->max_iter;
  const int kind = !bf16 ? 1 : (prm->refine_gap > 0.0 ? 3 : 2);
  bool graph = prm->use_graph != 0 && s != nullptr;
  if (iters == 0) {
    // nothing to iterate
  } else if (graph) {
    const bool reuse = c.graph_exec && c.graph_x == d_x && c.graph_atg == d_atg && c.graph_kind == kind &&
                       std::memcmp(&c.graph_prior, &pc, sizeof(PriorC)) == 0;
    if (!reuse) {
      if (c.graph_exec) {
        cudaGraphExecDestroy(c.graph_exec);
        c.graph_exec = nullptr;
      }
      if (int e = build_loop_graph(c, d_x, d_atg, pc, kind)) return e;
      c.graph_x = d_x;
      c.graph_atg = d_atg;
      c.graph_prior = pc;
      c.graph_kind = kind;
    }
    TMBIR_CUDA(cudaGraphLaunch(c.graph_exec, s));
  } else {
    if (int e = enqueue_iterations(c, d_x, d_atg, pc, iters, kind)) return e;
  }
  k_gather_final<<<1024, 256, 0, s>>>(c.state, d_x, c.xbuf[0], c.xbuf[1], c.total_voxels);
  TMBIR_CHECK_LAUNCH();
  k_rotation_reset<<<1, 1, 0, s>>>(c.state);
  TMBIR_CHECK_LAUNCH();
  c.state_ready = true;
  c.last_iters = iters;
  if (h_stats) {
    IterState st;
    TMBIR_CUDA(cudaMemcpyAsync(&st, c.state, sizeof(IterState), cudaMemcpyDeviceToHost, s));
    TMBIR_CUDA(cudaStreamSynchronize(s));
    h_stats->iterations = st.k;
    h_stats->restarts = st.restarts;
    h_stats->status = st.status;
    h_stats->objective = st.last_F;
    h_stats->gap = st.last_gap;
    h_stats->L = st.L;
    h_stats->grad_norm = std::sqrt(st.last_gg);
    c.last_iters = st.k;
    if (st.status != 0) return set_error(st.status, "reconstruct: non-finite value in a reduction");
  }
  return TMBIR_OK;
}

int tmbir_get_log(tmbir_ctx* ctx, double* h_log, int max_entries, int* n_out) {
  if (int e = require_ready(ctx, false)) return e;
  REQUIRE(h_log && n_out && max_entries >= 0, TMBIR_ERR_ARG, "get_log: NULL argument");
  Ctx& c = ctx->c;
  IterState st;
  TMBIR_CUDA(cudaMemcpyAsync(&st, c.state, sizeof(IterState), cudaMemcpyDeviceToHost, c.stream));
  TMBIR_CUDA(cudaStreamSynchronize(c.stream));
  const int n = std::min(std::min(st.k, max_entries), kLogCap);
  if (n > 0) {
    TMBIR_CUDA(cudaMemcpyAsync(h_log, c.log, (size_t)n * 4 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    TMBIR_CUDA(cudaStreamSynchronize(c.stream));
  }
  *n_out = n;
  return TMBIR_OK;
}

// one pass-1/2/3 sequence per group with explicit arguments, then the partial sums to the host
static int run_explicit(Ctx& c, const StepArgs& a, Pass3Mode m, const PriorC& pc, double* h_parts) {
  int off = 0;
  for (size_t i = 0; i < c.gdev.size(); ++i) {
    const GroupDev& g = c.gdev[i];
    if (int e = launch_convolution(g, a, m, pc, c.stream)) return e;
    if (int e = launch_pass3(g, a, m, pc, c.partials, off, c.stream, false, 2)) return e;
    off += blocks_pass3(g);
  }
  if (h_parts) {
    if (int e = launch_sum_partials(c.partials, off, c.dscal, c.stream)) return e;
    TMBIR_CUDA(cudaMemcpyAsync(h_parts, c.dscal, kParts * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    TMBIR_CUDA(cudaStreamSynchronize(c.stream));
  }
  return TMBIR_OK;
}

int tmbir_normal_apply(tmbir_ctx* ctx, const float* d_x, float* d_z) {
  TMBIR_TRACE("tmbir_normal_apply");
  if (int e = require_ready(ctx, true)) return e;
  REQUIRE(d_x && d_z && aligned16(d_x) && aligned16(d_z), TMBIR_ERR_ARG, "normal_apply: bad buffers");
  REQUIRE(d_x != d_z, TMBIR_ERR_ARG, "normal_apply: in-place not supported");
  StepArgs a{};
  a.x = d_x;
  a.xprev = d_x;
  a.beta = 0.f;
  a.out = d_z;
  PriorC pc{};
  return run_explicit(ctx->c, a, Pass3Mode::Apply, pc, nullptr);
}

int tmbir_gradient(tmbir_ctx* ctx, const float* d_x, const float* d_atg, const tmbir_params* prm, float* d_grad) {
  TMBIR_TRACE("tmbir_gradient");
  if (int e = require_ready(ctx, true)) return e;
  if (int e = check_params(prm)) return e;
  REQUIRE(d_x && d_atg && d_grad && aligned16(d_x) && aligned16(d_atg) && aligned16(d_grad), TMBIR_ERR_ARG,
          "gradient: bad buffers");
  REQUIRE(d_x != d_grad, TMBIR_ERR_ARG, "gradient: in-place not supported");
  StepArgs a{};
  a.x = d_x;
  a.xprev = d_x;
  a.beta = 0.f;
  a.atg = d_atg;
  a.out = d_grad;
  return run_explicit(ctx->c, a, Pass3Mode::Gradient, make_prior(*prm), nullptr);
}

int tmbir_step(tmbir_ctx* ctx, const float* d_x, const float* d_x_prev, double beta, const float* d_atg,
               const tmbir_params* prm, double L, float* d_x_next, double* h_partials) {
  TMBIR_TRACE("tmbir_step");
  if (int e = require_ready(ctx, true)) return e;
  if (int e = check_params(prm)) return e;
  REQUIRE(d_x && d_x_prev && d_atg && d_x_next && aligned16(d_x) && aligned16(d_x_prev) && aligned16(d_atg) &&
              aligned16(d_x_next),
          TMBIR_ERR_ARG, "step: bad buffers");
  REQUIRE(d_x_next != d_x && d_x_next != d_x_prev, TMBIR_ERR_ARG, "step: output must not alias the inputs");
  REQUIRE(L > 0.0 && std::isfinite(beta), TMBIR_ERR_ARG, "step: need L > 0 and finite beta");
  StepArgs a{};
  a.x = d_x;
  a.xprev = d_x_prev;
  a.beta = (float)beta;
  a.atg = d_atg;
  a.out = d_x_next;
  a.invL = (float)(1.0 / L);
  double parts[kParts];
  if (int e = run_explicit(ctx->c, a, Pass3Mode::Step, make_prior(*prm), parts)) return e;
  if (h_partials) std::memcpy(h_partials, parts, 5 * sizeof(double));
  return TMBIR_OK;
}

int tmbir_objective(tmbir_ctx* ctx, const float* d_x, const float* d_atg, const tmbir_params* prm, double* h_F) {
  TMBIR_TRACE("tmbir_objective");
  if (int e = require_ready(ctx, true)) return e;
  if (int e = check_params(prm)) return e;
  REQUIRE(d_x && d_atg && h_F && aligned16(d_x) && aligned16(d_atg), TMBIR_ERR_ARG, "objective: bad arguments");
  Ctx& c = ctx->c;
  StepArgs a{};
  a.x = d_x;
  a.xprev = d_x;
  a.beta = 0.f;
  a.atg = d_atg;
  a.out = nullptr;
  double parts[kParts];
  if (int e = run_explicit(c, a, Pass3Mode::Objective, make_prior(*prm), parts)) return e;
  double gh = 0.0;
  for (size_t i = 0; i < c.gdev.size(); ++i) {
    double v;
    TMBIR_CUDA(cudaMemcpy(&v, c.gdev[i].gtg, sizeof(double), cudaMemcpyDeviceToHost));
    gh += v;
  }
  *h_F = 0.5 * parts[0] - parts[1] + gh + prm->lambda * parts[2];
  return TMBIR_OK;
}

// ---------------------------------------------------------------- direct (non-Toeplitz) operators
static int ensure_spread(Ctx& c) {
  for (size_t i = 0; i < c.groups.size(); ++i)
    if (!c.spread_ready[i]) {
      if (int e = build_spread_matrix(c, (int)i)) return e;
      c.spread_ready[i] = true;
    }
  return TMBIR_OK;
}

int tmbir_forward(tmbir_ctx* ctx, const float* d_x, float* d_sino) {
  TMBIR_TRACE("tmbir_forward");
  if (int e = require_ready(ctx, false)) return e;
  REQUIRE(d_x && d_sino && aligned16(d_x) && aligned16(d_sino), TMBIR_ERR_ARG, "forward: bad buffers");
  Ctx& c = ctx->c;
  for (size_t i = 0; i < c.groups.size(); ++i)
    if (int e = forward_project(c, (int)i, d_x, d_sino)) return e;
  return TMBIR_OK;
}

int tmbir_adjoint(tmbir_ctx* ctx, const float* d_sino, float* d_x) {
  TMBIR_TRACE("tmbir_adjoint");
  if (int e = require_ready(ctx, false)) return e;
  REQUIRE(d_x && d_sino && aligned16(d_x) && aligned16(d_sino), TMBIR_ERR_ARG, "adjoint: bad buffers");
  Ctx& c = ctx->c;
  if (int e = ensure_spread(c)) return e;
  for (size_t i = 0; i < c.groups.size(); ++i)
    if (int e = backproject(c, (int)i, d_sino, d_x, false, false)) return e;
  return TMBIR_OK;
}

int tmbir_gradient_direct(tmbir_ctx* ctx, const float* d_x, const float* d_sino, const tmbir_params* prm,
                          float* d_grad, double* h_F) {
  TMBIR_TRACE("tmbir_gradient_direct");
  if (int e = require_ready(ctx, false)) return e;
  if (int e = check_params(prm)) return e;
  REQUIRE(d_x && d_sino && d_grad && aligned16(d_x) && aligned16(d_sino) && aligned16(d_grad), TMBIR_ERR_ARG,
          "gradient_direct: bad buffers");
  REQUIRE(d_x != d_grad, TMBIR_ERR_ARG, "gradient_direct: in-place not supported");
  Ctx& c = ctx->c;
  cudaStream_t s = c.stream;
  if (int e = ensure_spread(c)) return e;
  const int ng = (int)c.groups.size();
  // the residual r = R x - g in the sinogram domain, 1/2 r.r per group, R* r into each group's
  // K (*) y buffer; the data term enters pass 3b as that buffer against a zero R*g
  for (int i = 0; i < ng; ++i) {
    const GroupDev& g = c.gdev[i];
    if (int e = forward_project(c, i, d_x, c.sino_tmp)) return e;
    if (int e = residual(c, i, c.sino_tmp, d_sino)) return e;
    if (int e = half_sumsq(c, c.sino_tmp + g.sino_off, (size_t)g.S * g.na * g.nd, c.dscal + 16 + i, nullptr, g.wts,
                           g.na, g.nd))
      return e;
    if (int e = backproject(c, i, c.sino_tmp, g.kz, false, false, nullptr, nullptr, true, true)) return e;
  }
  TMBIR_CUDA(cudaMemsetAsync(c.xbuf[0], 0, c.total_voxels * sizeof(float), s));
  StepArgs a{};
  a.x = d_x;
  a.xprev = d_x;
  a.beta = 0.f;
  a.atg = c.xbuf[0];
  a.out = d_grad;
  const PriorC pc = make_prior(*prm);
  int off = 0;
  for (int i = 0; i < ng; ++i) {
    if (int e = launch_pass3(c.gdev[i], a, Pass3Mode::Gradient, pc, c.partials, off, s, false, 2)) return e;
    off += blocks_pass3(c.gdev[i]);
  }
  if (h_F) {
    // Phi(x) for the objective: the Gradient-mode stencil does not accumulate it, the Objective
    // mode does (its other partial sums are not used here)
    off = 0;
    for (int i = 0; i < ng; ++i) {
      if (int e = launch_pass3(c.gdev[i], a, Pass3Mode::Objective, pc, c.partials, off, s, false, 2)) return e;
      off += blocks_pass3(c.gdev[i]);
    }
    if (int e = launch_sum_partials(c.partials, off, c.dscal, s)) return e;
    std::vector<double> h(16 + ng);
    TMBIR_CUDA(cudaMemcpyAsync(h.data(), c.dscal, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    TMBIR_CUDA(cudaStreamSynchronize(s));
    double F = prm->lambda * h[2];
    for (int i = 0; i < ng; ++i) F += h[16 + i];
    *h_F = F;
  }
  return TMBIR_OK;
}

int tmbir_lambda_max(tmbir_ctx* ctx, double* h_out) {
  TMBIR_TRACE("tmbir_lambda_max");
  if (int e = require_ready(ctx, true)) return e;
  REQUIRE(h_out != nullptr, TMBIR_ERR_ARG, "lambda_max: NULL output");
  Ctx& c = ctx->c;
  TMBIR_CUDA(cudaStreamSynchronize(c.stream));
  for (size_t i = 0; i < c.gdev.size(); ++i)
    TMBIR_CUDA(cudaMemcpy(&h_out[i], c.gdev[i].lam_max, sizeof(double), cudaMemcpyDeviceToHost));
  return TMBIR_OK;
}

int tmbir_kernel(tmbir_ctx* ctx, int group, double* d_K) {
  if (int e = require_ready(ctx, true)) return e;
  Ctx& c = ctx->c;
  REQUIRE(group >= 0 && group < (int)c.gdev.size() && d_K != nullptr, TMBIR_ERR_ARG, "kernel: bad group or output");
  const size_t n = (size_t)(2 * c.gdev[group].N - 1) * (2 * c.gdev[group].N - 1);
  TMBIR_CUDA(cudaMemcpyAsync(d_K, c.gdev[group].K, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  return TMBIR_OK;
}

int tmbir_upsample_lanczos3(tmbir_ctx* ctx, const float* d_coarse, int n_slices, int Nc, float* d_fine) {
  TMBIR_TRACE("tmbir_upsample_lanczos3");
  REQUIRE(ctx != nullptr, TMBIR_ERR_ARG, "upsample: ctx is NULL");
  REQUIRE(d_coarse && d_fine && aligned16(d_coarse) && aligned16(d_fine), TMBIR_ERR_ARG, "upsample: bad buffers");
  REQUIRE(n_slices >= 0 && Nc >= 1 && Nc <= 1 << 15, TMBIR_ERR_ARG, "upsample: bad sizes");
  if (n_slices == 0) return TMBIR_OK;
  return launch_upsample_lanczos3(d_coarse, n_slices, Nc, d_fine, ctx->c.stream);
}

int tmbir_downsample_sino(tmbir_ctx* ctx, const float* d_sino, int n_slices, int n_angles, int n_det, int factor,
                          float* d_out) {
  TMBIR_TRACE("tmbir_downsample_sino");
  REQUIRE(ctx != nullptr, TMBIR_ERR_ARG, "downsample: ctx is NULL");
  REQUIRE(d_sino && d_out && aligned16(d_sino) && aligned16(d_out), TMBIR_ERR_ARG, "downsample: bad buffers");
  REQUIRE(n_slices >= 0 && n_angles >= 1 && n_det >= 2 && factor >= 1 && n_det % factor == 0 &&
              (n_det / factor) % 2 == 0,
          TMBIR_ERR_ARG, "downsample: need factor | n_det and an even coarse bin count");
  if (n_slices == 0) return TMBIR_OK;
  return launch_downsample_sino(d_sino, n_slices, n_angles, n_det, factor, d_out, ctx->c.stream);
}

int tmbir_pass_times(tmbir_ctx* ctx, float* d_x, const float* d_atg, const tmbir_params* prm, int iters, double* h_ms) {
  TMBIR_TRACE("tmbir_pass_times");
  if (int e = require_ready(ctx, true)) return e;
  if (int e = check_params(prm)) return e;
  REQUIRE(d_x && d_atg && h_ms && aligned16(d_x) && aligned16(d_atg) && iters >= 1 && iters <= kLogCap, TMBIR_ERR_ARG,
          "pass_times: bad arguments");
  Ctx& c = ctx->c;
  cudaStream_t s = c.stream;
  const PriorC pc = make_prior(*prm);
  const int ng = (int)c.gdev.size();
  for (int i = 0; i < ng; ++i) {
    TMBIR_CUDA(cudaMemcpyAsync(c.dscal + 16 + i, c.gdev[i].lam_max, sizeof(double), cudaMemcpyDeviceToDevice, s));
    TMBIR_CUDA(cudaMemcpyAsync(c.dscal + 16 + ng + i, c.gdev[i].gtg, sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  // the storage chosen by prm->spectra for every iteration (no refinement switch)
  const bool bf16 = prm->spectra == TMBIR_SPECTRA_BF16;
  k_init_state<<<1, 1, 0, s>>>(c.state, c.gmom, c.dscal + 16, c.dscal + 16 + ng, ng, prm->L, prm->lambda, prm->sigma,
                               prm->F_ref, 0.0, iters, prm->restart, bf16 ? 1 : 0, 0.0);
  TMBIR_CHECK_LAUNCH();
  TMBIR_CUDA(cudaMemcpyAsync(c.xbuf[1], d_x, c.total_voxels * sizeof(float), cudaMemcpyDeviceToDevice, s));
  StepArgs a{};
  a.atg = d_atg;
  a.xb[0] = d_x;
  a.xb[1] = c.xbuf[0];
  a.xb[2] = c.xbuf[1];
  a.st = c.state;
  // events between consecutive launches: passes 1, 2, 3a of every spectrum chunk, then 3b
  int max_chunks = 1;
  for (const GroupDev& g : c.gdev) max_chunks = std::max(max_chunks, (g.S + spec_chunk(g) - 1) / spec_chunk(g));
  std::vector<cudaEvent_t> ev(3 * max_chunks + 2);
  for (auto& e : ev) TMBIR_CUDA(cudaEventCreate(&e));
  auto span_ms = [&](int a0, int a1) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[a0], ev[a1]);
    return (double)ms;
  };
  double acc[5] = {0, 0, 0, 0, 0};
  int rc = TMBIR_OK;
  for (int k = 0; k < iters && rc == TMBIR_OK; ++k) {
    int off = 0;
    for (int i = 0; i < ng && rc == TMBIR_OK; ++i) {
      const GroupDev& g = c.gdev[i];
      a.gm = c.gmom + i;
      const int sc = spec_chunk(g), nch = (g.S + sc - 1) / sc;
      cudaEventRecord(ev[0], s);
      for (int ch = 0; ch < nch && rc == TMBIR_OK; ++ch) {
        const GroupDev v = chunk_view(g, ch * sc, std::min(sc, g.S - ch * sc));
        if ((rc = launch_pass1(v, a, s, bf16))) break;
        cudaEventRecord(ev[3 * ch + 1], s);
        if ((rc = launch_pass2(v, c.state, s, bf16))) break;
        cudaEventRecord(ev[3 * ch + 2], s);
        if ((rc = launch_pass3(v, a, Pass3Mode::Iterate, pc, nullptr, 0, s, bf16, 1))) break;
        cudaEventRecord(ev[3 * ch + 3], s);
      }
      if (rc) break;
      if ((rc = launch_pass3(g, a, Pass3Mode::Iterate, pc, c.partials, off, s, bf16, 2))) break;
      cudaEventRecord(ev[3 * nch + 1], s);
      cudaEventSynchronize(ev[3 * nch + 1]);
      for (int ch = 0; ch < nch; ++ch)
        for (int j = 0; j < 3; ++j) acc[j] += span_ms(3 * ch + j, 3 * ch + j + 1);
      acc[3] += span_ms(3 * nch, 3 * nch + 1);
      off += blocks_pass3(g);
    }
    if (rc) break;
    cudaEventRecord(ev[0], s);
    rc = launch_finalize(c.state, c.gmom, c.partials, group_blocks(c), c.log, s);
    cudaEventRecord(ev[1], s);
    cudaEventSynchronize(ev[1]);
    acc[4] += span_ms(0, 1);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  k_gather_final<<<1024, 256, 0, s>>>(c.state, d_x, c.xbuf[0], c.xbuf[1], c.total_voxels);
  TMBIR_CHECK_LAUNCH();
  k_rotation_reset<<<1, 1, 0, s>>>(c.state);
  TMBIR_CHECK_LAUNCH();
  c.state_ready = true;
  TMBIR_CUDA(cudaStreamSynchronize(s));
  for (int j = 0; j < 5; ++j) h_ms[j] = acc[j];
  return TMBIR_OK;
}

int tmbir_launch_count(const tmbir_ctx* ctx, long long* h_count) {
  REQUIRE(ctx != nullptr && h_count != nullptr, TMBIR_ERR_ARG, "launch_count: NULL argument");
  long long dev = 0;
  const Ctx& c = ctx->c;
  if (c.state) {
    // kernels run inside device-driven graph loops are counted on the device
    TMBIR_CUDA(cudaMemcpyAsync(&dev, &c.state->graph_launches, sizeof(long long), cudaMemcpyDeviceToHost, c.stream));
    TMBIR_CUDA(cudaStreamSynchronize(c.stream));
  }
  *h_count = __atomic_load_n(&g_launches, __ATOMIC_RELAXED) + dev;
  return TMBIR_OK;
}

// ---------------------------------------------------------------- autotuning

int tmbir_autotune(tmbir_ctx* ctx, const float* d_x, const float* d_atg, const tmbir_params* prm, int* h_zc,
                   int* h_sc) {
  TMBIR_TRACE("tmbir_autotune");
  if (int e = require_ready(ctx, true)) return e;
  if (int e = check_params(prm)) return e;
  REQUIRE(d_x && d_atg && aligned16(d_x) && aligned16(d_atg), TMBIR_ERR_ARG, "autotune: bad buffers");
  Ctx& c = ctx->c;
  cudaStream_t s = c.stream;
  const PriorC pc = make_prior(*prm);
  const int ng = (int)c.gdev.size();
  for (int i = 0; i < ng; ++i) {
    TMBIR_CUDA(cudaMemcpyAsync(c.dscal + 16 + i, c.gdev[i].lam_max, sizeof(double), cudaMemcpyDeviceToDevice, s));
    TMBIR_CUDA(cudaMemcpyAsync(c.dscal + 16 + ng + i, c.gdev[i].gtg, sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  // a state whose iterations never stop, and x_{-1} = x_0: pass 3 (Iterate) writes only the
  // rotation slot of x_{k+1} and the partial sums, never d_x
  k_init_state<<<1, 1, 0, s>>>(c.state, c.gmom, c.dscal + 16, c.dscal + 16 + ng, ng, prm->L, prm->lambda, prm->sigma,
                               0.0, 0.0, kLogCap, TMBIR_RESTART_GRADIENT, 0, 0.0);
  TMBIR_CHECK_LAUNCH();
  TMBIR_CUDA(cudaMemcpyAsync(c.xbuf[1], d_x, c.total_voxels * sizeof(float), cudaMemcpyDeviceToDevice, s));
  StepArgs a{};
  a.atg = d_atg;
  a.xb[0] = const_cast<float*>(d_x);
  a.xb[1] = c.xbuf[0];
  a.xb[2] = c.xbuf[1];
  a.st = c.state;
  cudaEvent_t e0, e1;
  TMBIR_CUDA(cudaEventCreate(&e0));
  TMBIR_CUDA(cudaEventCreate(&e1));
  int rc = TMBIR_OK;
  for (int i = 0; i < ng && rc == TMBIR_OK; ++i) {
    GroupDev& g = c.gdev[i];
    a.gm = c.gmom + i;
    // slices per spectrum chunk: passes 1, 2, 3a of the whole group with every candidate
    {
      std::vector<int> sc_c;
      for (int z : {4, 8, 16})
        if (z < g.S) sc_c.push_back(z);
      const int sc_d = g.S;  // one chunk
      sc_c.push_back(sc_d);
      float best = 1e30f;
      int best_sc = sc_d;
      for (int z : sc_c) {
        g.sc = z;
        float ms = 0.f;
        for (int rep = 0; rep < 3 && rc == TMBIR_OK; ++rep) {
          if (rep == 1) cudaEventRecord(e0, s);
          rc = launch_convolution(g, a, Pass3Mode::Iterate, pc, s);
        }
        if (rc) break;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rc = set_error(TMBIR_ERR_CUDA, "autotune: event timing failed");
          break;
        }
        if (ms < best) {
          best = ms;
          best_sc = z;
        }
      }
      if (rc) break;
      g.sc = best_sc;
      if (h_sc) h_sc[i] = best_sc;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned_sc[{g.N, g.S}] = best_sc;
    }
    // rows per block of passes 1 and 3a, where the side has variants (4 or 8 rows)
    if (g.N == 2048) {
      auto time_ms = [&](auto&& launch, float* out) {
        for (int rep = 0; rep < 3 && rc == TMBIR_OK; ++rep) {
          if (rep == 1) cudaEventRecord(e0, s);
          rc = launch();
        }
        if (rc) return;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(out, e0, e1) != cudaSuccess)
          rc = set_error(TMBIR_ERR_CUDA, "autotune: event timing failed");
      };
      float best1 = 1e30f, best3 = 1e30f;
      int rb1 = 4, rb3 = 8;
      for (int rb : {4, 8}) {
        float t1 = 0.f, t3 = 0.f;
        g.rb1 = g.rb3 = rb;
        time_ms([&] { return launch_pass1(g, a, s, false); }, &t1);
        time_ms([&] { return launch_pass3(g, a, Pass3Mode::Iterate, pc, nullptr, 0, s, false, 1); }, &t3);
        if (rc) break;
        if (t1 < best1) best1 = t1, rb1 = rb;
        if (t3 < best3) best3 = t3, rb3 = rb;
      }
      if (rc) break;
      g.rb1 = rb1;
      g.rb3 = rb3;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned_rb[{g.N, g.S}] = {rb1, rb3};
    }
    if ((rc = launch_convolution(g, a, Pass3Mode::Iterate, pc, s))) break;
    std::vector<int> cands;
    for (int z : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64})
      if (z <= g.S) cands.push_back(z);
    g.zc = 0;
    const int dflt = pass3_slices_per_block(g.S, pass3_row_blocks(g.N));
    if (std::find(cands.begin(), cands.end(), dflt) == cands.end()) cands.push_back(dflt);
    float best = 1e30f;
    int best_z = dflt;
    for (int z : cands) {
      g.zc = z;
      float ms = 0.f;
      for (int rep = 0; rep < 4 && rc == TMBIR_OK; ++rep) {
        if (rep == 1) cudaEventRecord(e0, s);
        rc = launch_pass3(g, a, Pass3Mode::Iterate, pc, c.partials, 0, s, false, 2);
      }
      if (rc) break;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = set_error(TMBIR_ERR_CUDA, "autotune: event timing failed");
        break;
      }
      if (ms < best) {
        best = ms;
        best_z = z;
      }
    }
    g.zc = best_z;
    if (h_zc) h_zc[i] = best_z;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned_zc[{g.N, g.S}] = best_z;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the block counts changed: the cached iteration graph and the run state are stale
  if (c.graph_exec) {
    cudaGraphExecDestroy(c.graph_exec);
    c.graph_exec = nullptr;
  }
  c.state_ready = false;
  return rc;
}

int tmbir_state_size(const tmbir_ctx* ctx, size_t* bytes) {
  if (int e = require_ready(ctx, false)) return e;
  REQUIRE(bytes != nullptr, TMBIR_ERR_ARG, "state_size: NULL argument");
  *bytes = state_header_bytes((int)ctx->c.groups.size()) + ctx->c.total_voxels * sizeof(float);
  return TMBIR_OK;
}

int tmbir_state_export(tmbir_ctx* ctx, void* d_state) {
  TMBIR_TRACE("tmbir_state_export");
  if (int e = require_ready(ctx, false)) return e;
  REQUIRE(d_state && aligned16(d_state), TMBIR_ERR_ARG, "state_export: buffer must be non-NULL and 16-byte aligned");
  Ctx& c = ctx->c;
  REQUIRE(c.state_ready, TMBIR_ERR_STATE, "state_export: no run to export");
  char* p = static_cast<char*>(d_state);
  const size_t ng = c.groups.size();
  TMBIR_CUDA(cudaMemcpyAsync(p, c.state, sizeof(IterState), cudaMemcpyDeviceToDevice, c.stream));
  TMBIR_CUDA(cudaMemcpyAsync(p + kStateHeader, c.gmom, ng * sizeof(GroupMom), cudaMemcpyDeviceToDevice, c.stream));
  TMBIR_CUDA(cudaMemcpyAsync(p + state_header_bytes((int)ng), c.xbuf[1], c.total_voxels * sizeof(float),
                             cudaMemcpyDeviceToDevice, c.stream));
  return TMBIR_OK;
}

int tmbir_state_import(tmbir_ctx* ctx, const void* d_state) {
  TMBIR_TRACE("tmbir_state_import");
  if (int e = require_ready(ctx, false)) return e;
  REQUIRE(d_state && aligned16(d_state), TMBIR_ERR_ARG, "state_import: buffer must be non-NULL and 16-byte aligned");
  Ctx& c = ctx->c;
  const char* p = static_cast<const char*>(d_state);
  // the device-side launch counter is the context's own, not part of the checkpoint
  long long launches = 0;
  TMBIR_CUDA(cudaMemcpyAsync(&launches, &c.state->graph_launches, sizeof(long long), cudaMemcpyDeviceToHost, c.stream));
  TMBIR_CUDA(cudaStreamSynchronize(c.stream));
  const size_t ng = c.groups.size();
  TMBIR_CUDA(cudaMemcpyAsync(c.state, p, sizeof(IterState), cudaMemcpyDeviceToDevice, c.stream));
  TMBIR_CUDA(cudaMemcpyAsync(&c.state->graph_launches, &launches, sizeof(long long), cudaMemcpyHostToDevice, c.stream));
  TMBIR_CUDA(cudaMemcpyAsync(c.gmom, p + kStateHeader, ng * sizeof(GroupMom), cudaMemcpyDeviceToDevice, c.stream));
  TMBIR_CUDA(cudaMemcpyAsync(c.xbuf[1], p + state_header_bytes((int)ng), c.total_voxels * sizeof(float),
                             cudaMemcpyDeviceToDevice, c.stream));
  TMBIR_CUDA(cudaStreamSynchronize(c.stream));
  c.state_ready = true;
  return TMBIR_OK;
}

int tmbir_sync(tmbir_ctx* ctx) {
  REQUIRE(ctx != nullptr, TMBIR_ERR_ARG, "sync: ctx is NULL");
  TMBIR_CUDA(cudaStreamSynchronize(ctx->c.stream));
  TMBIR_CUDA(cudaGetLastError());
  return TMBIR_OK;
}

}  // extern "C"
