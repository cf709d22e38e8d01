// tmbir_wait_check: the give-up path of the library's bounded device waits, testable without
// faulting or hanging a GPU.  Every wait of the library on a barrier polls a bounded number of
// times (the tensor-core convolutions wait on their MMAs this way) and, when it gives up, records
// that in a status word and lets the kernel return, so the host reports TMBIR_ERR_TIMEOUT and the
// context stays usable.  Here one block waits on a shared-memory mbarrier that nothing arrives
// on (arrive = 0), or that one of its threads arrives on first (arrive = 1).
#include "internal.h"
#include "tc05.cuh"

namespace tmbir {

// 0: the last check's wait completed, 1: it gave up
static __device__ int g_wait_status;

__global__ void k_wait_check(uint32_t polls, int arrive) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc05::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) tc05::mbar_arrive(&bar);
  const bool ok = tc05::mbar_wait(&bar, 0u, polls);
  // every thread has stopped waiting once this barrier passes
  const int gave_up = __syncthreads_or(!ok);
  if (threadIdx.x == 0) {
    tc05::mbar_inval(&bar);
    g_wait_status = gave_up ? 1 : 0;
  }
}

}  // namespace tmbir

using namespace tmbir;

extern "C" int tmbir_wait_check(tmbir_ctx* ctx, unsigned polls, int arrive) {
  TMBIR_TRACE("tmbir_wait_check");
  if (!ctx) return set_error(TMBIR_ERR_ARG, "wait_check: ctx is NULL");
  if (polls < 1u || polls > (1u << 24)) return set_error(TMBIR_ERR_ARG, "wait_check: polls must be in [1, 2^24]");
  Ctx& c = ctx->c;
  k_wait_check<<<1, 64, 0, c.stream>>>(polls, arrive ? 1 : 0);
  TMBIR_CHECK_LAUNCH();
  int gave_up = 0;
  TMBIR_CUDA(cudaMemcpyFromSymbolAsync(&gave_up, g_wait_status, sizeof(int), 0, cudaMemcpyDeviceToHost, c.stream));
  TMBIR_CUDA(cudaStreamSynchronize(c.stream));
  if (gave_up) return set_error(TMBIR_ERR_TIMEOUT, "wait_check: the bounded device wait gave up");
  return TMBIR_OK;
}
