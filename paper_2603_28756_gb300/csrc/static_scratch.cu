// tmbir_normal_apply_static: the normal operator of tmbir_normal_apply with its scratch memory
// (the intermediate half spectra and the per-block partial sums) in a fixed-size array that is
// part of the library image, for callers that cannot allocate device memory when they call.
//
// The array is a file-scope __device__ variable: every device that loads the library holds it
// until the process exits.  Host code only sees a host-side stand-in for its name, so the
// device address is looked up with cudaGetSymbolAddress while the device is current.  The
// lookup loads this file's module, which commits the arrays' device memory; tmbir_create does
// it for the device current at creation (and refreshes the cached address each time, so a
// context created after a device reset sees the new address), and the entry point itself does
// it for a device that has no context yet.
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace tmbir {

// 8 Mi complex floats (64 MiB) of half spectra: for example 7 slices of 1024^2, or 31 of 512^2
// at once; the passes run in chunks of slices that fit
constexpr size_t kStaticSpecElems = (size_t)8 << 20;
// partial sums of up to 65536 reducing blocks
constexpr size_t kStaticPartElems = (size_t)65536 * kParts;

static __device__ __align__(256) float2 g_static_spec[kStaticSpecElems];
static __device__ __align__(256) double g_static_parts[kStaticPartElems];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
float2* g_spec_addr[kMaxDevices] = {};
double* g_part_addr[kMaxDevices] = {};

int current_device(int* dev) {
  TMBIR_CUDA(cudaGetDevice(dev));
  if (*dev < 0 || *dev >= kMaxDevices) return set_error(TMBIR_ERR_CUDA, "static scratch: device index out of range");
  return TMBIR_OK;
}

// looks the two arrays up on the current device (the caller holds g_static_mu)
int lookup_locked(int dev) {
  void* p = nullptr;
  void* q = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_spec);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_static_parts);
  if (e != cudaSuccess)
    return set_error(TMBIR_ERR_CUDA, std::string("static scratch: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  g_spec_addr[dev] = static_cast<float2*>(p);
  g_part_addr[dev] = static_cast<double*>(q);
  return TMBIR_OK;
}
}  // namespace

int static_scratch_resolve() {
  int dev = 0;
  if (int e = current_device(&dev)) return e;
  std::lock_guard<std::mutex> lock(g_static_mu);
  return lookup_locked(dev);
}

// device addresses of the two arrays on the current device (looked up on first use)
static int static_scratch(float2** spec, double** parts) {
  int dev = 0;
  if (int e = current_device(&dev)) return e;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_spec_addr[dev])
    if (int e = lookup_locked(dev)) return e;
  *spec = g_spec_addr[dev];
  *parts = g_part_addr[dev];
  return TMBIR_OK;
}

}  // namespace tmbir

using namespace tmbir;

extern "C" int tmbir_normal_apply_static(tmbir_ctx* ctx, const float* d_x, float* d_z) {
  TMBIR_TRACE("tmbir_normal_apply_static");
  if (int e = require_ready(ctx, true)) return e;
  Ctx& c = ctx->c;
  if (!d_x || !d_z || ((uintptr_t)d_x & 15u) || ((uintptr_t)d_z & 15u) || d_x == d_z)
    return set_error(TMBIR_ERR_ARG, "normal_apply_static: bad buffers");
  // the groups one after another, each in spectrum chunks that fit the static array
  int blocks = 0;
  for (const GroupDev& g : c.gdev) {
    const size_t per = (size_t)(g.N + 1) * g.N;
    if (per > kStaticSpecElems)
      return set_error(TMBIR_ERR_SHAPE, "normal_apply_static: one slice needs " + std::to_string(per) +
                                            " complex scratch values, the static array holds " +
                                            std::to_string(kStaticSpecElems));
    blocks += blocks_pass3(g);
  }
  if ((size_t)blocks * kParts > kStaticPartElems)
    return set_error(TMBIR_ERR_SHAPE, "normal_apply_static: too many reducing blocks for the static array");
  float2* spec = nullptr;
  double* parts = nullptr;
  if (int e = static_scratch(&spec, &parts)) return e;
  StepArgs a{};
  a.x = d_x;
  a.xprev = d_x;
  a.beta = 0.f;
  a.out = d_z;
  PriorC pc{};
  int boff = 0;
  for (const GroupDev& g0 : c.gdev) {
    GroupDev g = g0;
    g.spec = spec;
    g.sc = std::min(spec_chunk(g0), (int)(kStaticSpecElems / ((size_t)(g.N + 1) * g.N)));
    if (int e = launch_convolution(g, a, Pass3Mode::Apply, pc, c.stream)) return e;
    if (int e = launch_pass3(g, a, Pass3Mode::Apply, pc, parts, boff, c.stream, false, 2)) return e;
    boff += blocks_pass3(g);
  }
  return TMBIR_OK;
}
