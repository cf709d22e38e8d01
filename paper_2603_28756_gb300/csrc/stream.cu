// Volumes larger than the device's memory (Sec. 2.4).  The volume, its sinogram and R*g stay in
// host memory (R*g may instead stay in device memory, read in place) and pass through the GPU in
// slabs of slices; the context's one geometry group is the slab.  The paper's node scheduler (three threads joined by bounded work queues: copies in,
// kernels, copies out) becomes three CUDA streams and two device buffer sets ordered by events,
// so the copies of slab j + 1 in and of slab j - 1 out overlap the kernels of slab j.
//
// Every slab runs the kernels of a resident volume.  Pass 3b of a slab sees one halo slice on
// each side (the 26-neighbourhood crosses slab boundaries, Sec. 2.4's halo) and computes only the
// slab's own slices; its blocks write their partial sums at the rows a resident volume's blocks of
// the same slices use, and the finalize kernel reduces all slabs' rows in that order.  With a slab
// that is a multiple of the slices per pass-3b block the iterates are those of the resident
// volume bit for bit.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace tmbir {
namespace {

#define SREQ(cond, code, msg)                   \
  do {                                          \
    if (!(cond)) return set_error(code, msg);   \
  } while (0)

// Carve-up of the caller's device buffer for a volume of n slices.
struct Plan {
  int N = 0, slab = 0, n = 0, zc = 0, nb = 0, nslab = 0;
  size_t img = 0;   // floats of one slab image buffer: slab + 2 halo slices
  size_t sino = 0;  // floats of one slab sinogram
  size_t off_x[2], off_xp[2], off_atg[2], off_out[2], off_sino[2], off_kz, off_part, off_gtg, bytes;
};

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// zc: slices per pass-3b block (0: the bound of any choice, one slice per block)
int make_plan(const Ctx& c, int n_slices, int zc, Plan* p) {
  SREQ(c.groups.size() == 1, TMBIR_ERR_ARG, "stream: the context must hold exactly one group (the slab)");
  SREQ(n_slices >= 1, TMBIR_ERR_ARG, "stream: n_slices must be >= 1");
  const tmbir_group& g = c.groups[0];
  p->N = g.N;
  p->slab = g.n_slices;
  p->n = n_slices;
  p->nslab = (n_slices + p->slab - 1) / p->slab;
  p->nb = pass3_row_blocks(g.N);
  p->zc = zc;
  const size_t N2 = (size_t)g.N * g.N;
  p->img = (size_t)(p->slab + 2) * N2;
  p->sino = (size_t)p->slab * g.n_angles * g.n_det;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = up256(off);
    off = o + bytes;
    return o;
  };
  for (int s = 0; s < 2; ++s) {
    p->off_x[s] = take(p->img * sizeof(float));
    p->off_xp[s] = take(p->img * sizeof(float));
    p->off_atg[s] = take(p->img * sizeof(float));
    p->off_out[s] = take(p->img * sizeof(float));
    p->off_sino[s] = take(p->sino * sizeof(float));
  }
  p->off_kz = take(p->img * sizeof(float));
  const int zc_min = zc > 0 ? zc : 1;
  p->off_part = take((size_t)p->nb * ((n_slices + zc_min - 1) / zc_min) * kParts * sizeof(double));
  p->off_gtg = take((size_t)p->nslab * sizeof(double));
  p->bytes = up256(off);
  return TMBIR_OK;
}

// the slices per pass-3b block of a run: the slab's rule (or tuned value), lowered until it
// divides the slab so that every slab but the last covers whole blocks
int run_zc(const Ctx& c) {
  const GroupDev& g = c.gdev[0];
  int zc = pass3_zc(g, pass3_row_blocks(g.N));
  while (zc > 1 && g.S % zc) --zc;
  return zc;
}

int ensure_streams(Ctx& c) {
  if (c.s_in) return TMBIR_OK;
  TMBIR_CUDA(cudaStreamCreateWithFlags(&c.s_in, cudaStreamNonBlocking));
  TMBIR_CUDA(cudaStreamCreateWithFlags(&c.s_out, cudaStreamNonBlocking));
  for (int s = 0; s < 2; ++s) {
    TMBIR_CUDA(cudaEventCreateWithFlags(&c.ev_in[s], cudaEventDisableTiming));
    TMBIR_CUDA(cudaEventCreateWithFlags(&c.ev_comp[s], cudaEventDisableTiming));
    TMBIR_CUDA(cudaEventCreateWithFlags(&c.ev_out[s], cudaEventDisableTiming));
  }
  TMBIR_CUDA(cudaEventCreateWithFlags(&c.ev_start, cudaEventDisableTiming));
  return TMBIR_OK;
}

// the copy streams start after the work already on the context stream
int fork_copies(Ctx& c) {
  TMBIR_CUDA(cudaEventRecord(c.ev_start, c.stream));
  TMBIR_CUDA(cudaStreamWaitEvent(c.s_in, c.ev_start, 0));
  TMBIR_CUDA(cudaStreamWaitEvent(c.s_out, c.ev_start, 0));
  return TMBIR_OK;
}

// wait for all three streams (also after an error, so no copy outlives the call)
int join_all(Ctx& c, int rc) {
  const cudaError_t a = cudaStreamSynchronize(c.s_in);
  const cudaError_t b = cudaStreamSynchronize(c.stream);
  const cudaError_t d = cudaStreamSynchronize(c.s_out);
  if (rc) return rc;
  if (a != cudaSuccess || b != cudaSuccess || d != cudaSuccess)
    return set_error(TMBIR_ERR_CUDA, std::string("stream: ") +
                                         cudaGetErrorString(a != cudaSuccess ? a : (b != cudaSuccess ? b : d)));
  return TMBIR_OK;
}

int check_common(tmbir_ctx* ctx, int n_slices, const void* d_swork, size_t swork_bytes, Plan* p, int zc) {
  if (int e = require_ready(ctx, false)) return e;
  Ctx& c = ctx->c;
  SREQ(c.stream != nullptr, TMBIR_ERR_ARG, "stream: needs a context stream (not the legacy stream)");
  if (int e = make_plan(c, n_slices, zc, p)) return e;
  SREQ(d_swork != nullptr && ((uintptr_t)d_swork & 255u) == 0, TMBIR_ERR_ARG,
       "stream: device buffer must be non-NULL and 256-byte aligned");
  SREQ(swork_bytes >= p->bytes, TMBIR_ERR_WORKSPACE, "stream: device buffer too small");
  return ensure_streams(c);
}

// one slab's build: R*g (and the FBP start) of slices [a, a + n) from the sinogram in set s
int build_slab(tmbir_ctx* ctx, const Plan& p, char* ws, int j, int s, float* h_atg, float* h_x0) {
  Ctx& c = ctx->c;
  const tmbir_group& g = c.groups[0];
  const int a = j * p.slab, n = std::min(p.slab, p.n - a);
  const size_t N2 = (size_t)p.N * p.N;
  float* d_sino = reinterpret_cast<float*>(ws + p.off_sino[s]);
  float* d_atg = reinterpret_cast<float*>(ws + p.off_atg[s]);
  float* d_x0 = reinterpret_cast<float*>(ws + p.off_out[s]);
  TMBIR_CUDA(cudaStreamWaitEvent(c.stream, c.ev_in[s], 0));   // the slab's sinogram is in
  TMBIR_CUDA(cudaStreamWaitEvent(c.stream, c.ev_out[s], 0));  // set s's outputs are copied out
  if (n < p.slab)  // a short last slab: zero slices add nothing to 1/2 g.g
    TMBIR_CUDA(cudaMemsetAsync(d_sino + (size_t)n * g.n_angles * g.n_det, 0,
                               (size_t)(p.slab - n) * g.n_angles * g.n_det * sizeof(float), c.stream));
  if (h_x0) {
    if (int e = tmbir_build_operator_fbp(ctx, d_sino, d_atg, d_x0)) return e;
  } else {
    if (int e = tmbir_build_operator(ctx, d_sino, d_atg)) return e;
  }
  TMBIR_CUDA(cudaMemcpyAsync(reinterpret_cast<double*>(ws + p.off_gtg) + j, c.gdev[0].gtg, sizeof(double),
                             cudaMemcpyDeviceToDevice, c.stream));
  TMBIR_CUDA(cudaEventRecord(c.ev_comp[s], c.stream));
  TMBIR_CUDA(cudaStreamWaitEvent(c.s_out, c.ev_comp[s], 0));
  TMBIR_CUDA(cudaMemcpyAsync(h_atg + (size_t)a * N2, d_atg, (size_t)n * N2 * sizeof(float), cudaMemcpyDeviceToHost,
                             c.s_out));
  if (h_x0)
    TMBIR_CUDA(cudaMemcpyAsync(h_x0 + (size_t)a * N2, d_x0, (size_t)n * N2 * sizeof(float), cudaMemcpyDeviceToHost,
                               c.s_out));
  TMBIR_CUDA(cudaEventRecord(c.ev_out[s], c.s_out));
  return TMBIR_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int sino_in(Ctx& c, const Plan& p, char* ws, int j, const float* h_sino) {
  const tmbir_group& g = c.groups[0];
  const int s = j & 1, a = j * p.slab, n = std::min(p.slab, p.n - a);
  const size_t per = (size_t)g.n_angles * g.n_det;
  TMBIR_CUDA(cudaStreamWaitEvent(c.s_in, c.ev_comp[s], 0));  // the build of slab j - 2 has read set s
  TMBIR_CUDA(cudaMemcpyAsync(ws + p.off_sino[s], h_sino + (size_t)a * per, (size_t)n * per * sizeof(float),
                             cudaMemcpyHostToDevice, c.s_in));
  TMBIR_CUDA(cudaEventRecord(c.ev_in[s], c.s_in));
  return TMBIR_OK;
}

// Slab j of an iteration: volume slices [a, a + n) with halo slices a - 1 (lo) and a + n (hi)
// where they exist; device buffers of set j & 1 hold volume slices a - lo .. a + n + hi - 1.
struct SlabGeo {
  int a, n, lo, hi;
};
SlabGeo slab_geo(const Plan& p, int j) {
  SlabGeo q;
  q.a = j * p.slab;
  q.n = std::min(p.slab, p.n - q.a);
  q.lo = q.a > 0 ? 1 : 0;
  q.hi = q.a + q.n < p.n ? 1 : 0;
  return q;
}

// copies in of slab j: x_k and x_{k-1} with the halo, and R*g of the slab's own slices (unless R*g
// is in device memory)
int iter_in(Ctx& c, const Plan& p, char* ws, int j, const float* xk, const float* xkm1, const float* h_atg,
            bool atg_dev) {
  const int s = j & 1;
  const SlabGeo q = slab_geo(p, j);
  const size_t N2 = (size_t)p.N * p.N;
  const size_t first = (size_t)(q.a - q.lo) * N2, cnt = (size_t)(q.n + q.lo + q.hi) * N2;
  TMBIR_CUDA(cudaStreamWaitEvent(c.s_in, c.ev_comp[s], 0));  // slab j - 2's kernels are done with set s
  TMBIR_CUDA(cudaMemcpyAsync(ws + p.off_x[s], xk + first, cnt * sizeof(float), cudaMemcpyHostToDevice, c.s_in));
  TMBIR_CUDA(cudaMemcpyAsync(ws + p.off_xp[s], xkm1 + first, cnt * sizeof(float), cudaMemcpyHostToDevice, c.s_in));
  if (!atg_dev)
    TMBIR_CUDA(cudaMemcpyAsync(reinterpret_cast<float*>(ws + p.off_atg[s]) + (size_t)q.lo * N2,
                               h_atg + (size_t)q.a * N2, (size_t)q.n * N2 * sizeof(float), cudaMemcpyHostToDevice,
                               c.s_in));
  TMBIR_CUDA(cudaEventRecord(c.ev_in[s], c.s_in));
  return TMBIR_OK;
}

// the kernels of slab j in Iterate mode, both storage variants of `kind` (each checks the run's
// phase on the device, as in tmbir_reconstruct)
int iter_compute(Ctx& c, const Plan& p, char* ws, int j, int cur, const PriorC& pc, int kind, const float* d_atg) {
  const int s = j & 1;
  const SlabGeo q = slab_geo(p, j);
  TMBIR_CUDA(cudaStreamWaitEvent(c.stream, c.ev_in[s], 0));
  TMBIR_CUDA(cudaStreamWaitEvent(c.stream, c.ev_out[s], 0));  // slab j - 2's x_{k+1} has left set s
  GroupDev v = c.gdev[0];
  v.S = q.n + q.lo + q.hi;
  v.zlo = q.lo;
  v.zn = q.n;
  v.zc = p.zc;
  v.slice0 = 0;
  v.img_off = 0;
  v.kz = reinterpret_cast<float*>(ws + p.off_kz);
  StepArgs a{};
  // R*g at the slab's buffer index z: the set's copy, or the device volume from slice a - lo
  a.atg = d_atg ? d_atg + (size_t)(q.a - q.lo) * p.N * p.N : reinterpret_cast<const float*>(ws + p.off_atg[s]);
  a.xb[cur] = reinterpret_cast<float*>(ws + p.off_x[s]);
  a.xb[(cur + 2) % 3] = reinterpret_cast<float*>(ws + p.off_xp[s]);
  a.xb[(cur + 1) % 3] = reinterpret_cast<float*>(ws + p.off_out[s]);
  a.st = c.state;
  a.gm = c.gmom;
  double* partials = reinterpret_cast<double*>(ws + p.off_part);
  const int off = (q.a / p.zc) * p.nb;
  const GroupDev own = chunk_view(v, q.lo, q.n);  // passes 1, 2, 3a: the slab's own slices
  for (int variant = 0; variant < 2; ++variant) {
    const bool bf16 = variant == 0;
    if (bf16 ? kind < 2 : kind == 2) continue;
    if (int e = launch_convolution(own, a, Pass3Mode::Iterate, pc, c.stream, bf16)) return e;
    if (int e = launch_pass3(v, a, Pass3Mode::Iterate, pc, partials, off, c.stream, bf16, 2)) return e;
  }
  TMBIR_CUDA(cudaEventRecord(c.ev_comp[s], c.stream));
  return TMBIR_OK;
}

// copies out of slab j: x_{k+1} of its own slices, into the host slot that held x_{k-2} (three
// slots rotate, so no copy in of this iteration reads it)
int iter_out(Ctx& c, const Plan& p, char* ws, int j, float* xnext) {
  const int s = j & 1;
  const SlabGeo q = slab_geo(p, j);
  const size_t N2 = (size_t)p.N * p.N;
  TMBIR_CUDA(cudaStreamWaitEvent(c.s_out, c.ev_comp[s], 0));
  TMBIR_CUDA(cudaMemcpyAsync(xnext + (size_t)q.a * N2, reinterpret_cast<float*>(ws + p.off_out[s]) + (size_t)q.lo * N2,
                             (size_t)q.n * N2 * sizeof(float), cudaMemcpyDeviceToHost, c.s_out));
  TMBIR_CUDA(cudaEventRecord(c.ev_out[s], c.s_out));
  return TMBIR_OK;
}

// the final iterate from host slot src into the caller's buffer dst, slab by slab through the
// device (copies in and out overlap; a host-to-host copy runs far below the link's rate)
int copy_back(Ctx& c, const Plan& p, char* ws, const float* src, float* dst) {
  const size_t N2 = (size_t)p.N * p.N;
  for (int j = 0; j < p.nslab; ++j) {
    const int s = j & 1, a = j * p.slab, n = std::min(p.slab, p.n - a);
    TMBIR_CUDA(cudaStreamWaitEvent(c.s_in, c.ev_out[s], 0));  // set s's previous slab has left
    TMBIR_CUDA(cudaMemcpyAsync(ws + p.off_x[s], src + (size_t)a * N2, (size_t)n * N2 * sizeof(float),
                               cudaMemcpyHostToDevice, c.s_in));
    TMBIR_CUDA(cudaEventRecord(c.ev_in[s], c.s_in));
    TMBIR_CUDA(cudaStreamWaitEvent(c.s_out, c.ev_in[s], 0));
    TMBIR_CUDA(cudaMemcpyAsync(dst + (size_t)a * N2, ws + p.off_x[s], (size_t)n * N2 * sizeof(float),
                               cudaMemcpyDeviceToHost, c.s_out));
    TMBIR_CUDA(cudaEventRecord(c.ev_out[s], c.s_out));
  }
  return TMBIR_OK;
}

}  // namespace
}  // namespace tmbir

using namespace tmbir;

extern "C" {

int tmbir_stream_workspace_size(const tmbir_ctx* ctx, int n_slices, size_t* bytes) {
  SREQ(ctx != nullptr && bytes != nullptr, TMBIR_ERR_ARG, "stream_workspace_size: NULL argument");
  SREQ(!ctx->c.groups.empty(), TMBIR_ERR_STATE, "stream_workspace_size: no geometry");
  Plan p;
  if (int e = make_plan(ctx->c, n_slices, 0, &p)) return e;
  *bytes = p.bytes;
  return TMBIR_OK;
}

int tmbir_stream_build_operator(tmbir_ctx* ctx, int n_slices, const float* h_sino, float* h_atg, float* h_x0,
                                void* d_swork, size_t swork_bytes, double* h_gtg) {
  TMBIR_TRACE("tmbir_stream_build_operator");
  Plan p;
  if (int e = check_common(ctx, n_slices, d_swork, swork_bytes, &p, 0)) return e;
  SREQ(h_sino && h_atg && h_gtg, TMBIR_ERR_ARG, "stream_build_operator: NULL host buffer");
  SREQ(h_x0 != h_atg, TMBIR_ERR_ARG, "stream_build_operator: R*g and the start must be different buffers");
  Ctx& c = ctx->c;
  char* ws = static_cast<char*>(d_swork);
  int rc = fork_copies(c);
  if (!rc) rc = sino_in(c, p, ws, 0, h_sino);
  for (int j = 0; j < p.nslab && !rc; ++j) {
    if (j + 1 < p.nslab) rc = sino_in(c, p, ws, j + 1, h_sino);
    if (!rc) rc = build_slab(ctx, p, ws, j, j & 1, h_atg, h_x0);
  }
  std::vector<double> gtg(p.nslab, 0.0);
  if (!rc)
    if (cudaMemcpyAsync(gtg.data(), ws + p.off_gtg, p.nslab * sizeof(double), cudaMemcpyDeviceToHost, c.stream) !=
        cudaSuccess)
      rc = set_error(TMBIR_ERR_CUDA, "stream_build_operator: reading 1/2 g.g");
  rc = join_all(c, rc);
  if (rc) return rc;
  double sum = 0.0;
  for (double v : gtg) sum += v;  // slab order
  *h_gtg = sum;
  return TMBIR_OK;
}

int tmbir_stream_reconstruct(tmbir_ctx* ctx, int n_slices, float* h_x, const float* atg, double gtg_half,
                             float* h_work, void* d_swork, size_t swork_bytes, const tmbir_params* prm,
                             tmbir_stats* h_stats) {
  TMBIR_TRACE("tmbir_stream_reconstruct");
  if (int e = require_ready(ctx, true)) return e;
  if (int e = check_params(prm)) return e;
  SREQ(!prm->resume, TMBIR_ERR_ARG, "stream_reconstruct: resume is not supported for host volumes");
  SREQ(prm->max_iter >= 0 && prm->max_iter <= kLogCap, TMBIR_ERR_ARG, "stream_reconstruct: max_iter out of range");
  SREQ(h_x && atg && h_work, TMBIR_ERR_ARG, "stream_reconstruct: NULL buffer");
  SREQ(std::isfinite(gtg_half) && gtg_half >= 0.0, TMBIR_ERR_ARG, "stream_reconstruct: gtg_half must be >= 0");
  Ctx& c = ctx->c;
  const int zc = run_zc(c);
  Plan p;
  if (int e = check_common(ctx, n_slices, d_swork, swork_bytes, &p, zc)) return e;
  char* ws = static_cast<char*>(d_swork);
  // R*g in device memory stays there; only the iterates stream
  cudaPointerAttributes pa{};
  TMBIR_CUDA(cudaPointerGetAttributes(&pa, atg));
  const bool atg_dev = pa.type == cudaMemoryTypeDevice;
  SREQ(!atg_dev || aligned16(atg), TMBIR_ERR_ARG, "stream_reconstruct: device R*g must be 16-byte aligned");
  const PriorC pc = make_prior(*prm);
  const bool bf16 = prm->spectra == TMBIR_SPECTRA_BF16;
  const int kind = !bf16 ? 1 : (prm->refine_gap > 0.0 ? 3 : 2);
  cudaStream_t s = c.stream;
  // the step constant from this geometry's lambda_max, 1/2 g.g of the whole volume
  TMBIR_CUDA(cudaMemcpyAsync(c.dscal + 16, c.gdev[0].lam_max, sizeof(double), cudaMemcpyDeviceToDevice, s));
  TMBIR_CUDA(cudaMemcpyAsync(c.dscal + 17, &gtg_half, sizeof(double), cudaMemcpyHostToDevice, s));
  if (int e = launch_init_state(c, *prm, c.dscal + 16, c.dscal + 17, 1, s)) return e;
  c.state_ready = false;  // the rotation lives on the host: nothing to export or resume
  float* slot[3] = {h_x, h_work, h_work + (size_t)n_slices * p.N * p.N};
  const GroupBlocks gb{1, {0, p.nb * ((n_slices + p.zc - 1) / p.zc)}};
  int cur = 0, rc = TMBIR_OK;
  IterState st{};
  for (int k = 0; k < prm->max_iter && !rc; ++k) {
    const float* xk = slot[cur];
    const float* xkm1 = k == 0 ? slot[cur] : slot[(cur + 2) % 3];  // x_{-1} = x_0
    float* xnext = slot[(cur + 1) % 3];
    rc = fork_copies(c);
    if (!rc) rc = iter_in(c, p, ws, 0, xk, xkm1, atg, atg_dev);
    for (int j = 0; j < p.nslab && !rc; ++j) {
      if (j + 1 < p.nslab) rc = iter_in(c, p, ws, j + 1, xk, xkm1, atg, atg_dev);
      if (!rc) rc = iter_compute(c, p, ws, j, cur, pc, kind, atg_dev ? atg : nullptr);
      if (!rc) rc = iter_out(c, p, ws, j, xnext);
    }
    if (!rc) rc = launch_finalize(c.state, c.gmom, reinterpret_cast<double*>(ws + p.off_part), gb, c.log, s);
    if (!rc && cudaMemcpyAsync(&st, c.state, sizeof(IterState), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      rc = set_error(TMBIR_ERR_CUDA, "stream_reconstruct: reading the state");
    rc = join_all(c, rc);
    if (rc) break;
    cur = st.cur;
    if (st.done) break;
  }
  if (rc) return rc;
  if (prm->max_iter == 0) {  // no iteration: the state as initialised
    TMBIR_CUDA(cudaMemcpyAsync(&st, c.state, sizeof(IterState), cudaMemcpyDeviceToHost, s));
    TMBIR_CUDA(cudaStreamSynchronize(s));
  }
  if (prm->max_iter > 0 && cur != 0) {  // the final iterate back into the caller's buffer
    rc = fork_copies(c);
    if (!rc) rc = copy_back(c, p, ws, slot[cur], h_x);
    if ((rc = join_all(c, rc))) return rc;
  }
  c.last_iters = st.k;
  if (h_stats) {
    h_stats->iterations = st.k;
    h_stats->restarts = st.restarts;
    h_stats->status = st.status;
    h_stats->objective = st.last_F;
    h_stats->gap = st.last_gap;
    h_stats->L = st.L;
    h_stats->grad_norm = std::sqrt(st.last_gg);
  }
  if (st.status != 0) return set_error(st.status, "stream_reconstruct: non-finite value in a reduction");
  return TMBIR_OK;
}

}  // extern "C"
