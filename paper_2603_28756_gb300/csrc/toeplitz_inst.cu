// Instantiates the three Toeplitz passes for one image side N (compiled once per supported N
// with -DTMBIR_N=<N>, so the sizes build in parallel).
#include "toeplitz_kernels.cuh"

#ifndef TMBIR_N
#error "compile with -DTMBIR_N=<image side>"
#endif

#define TMBIR_CAT2(a, b) a##b
#define TMBIR_CAT(a, b) TMBIR_CAT2(a, b)

namespace tmbir {
int TMBIR_CAT(pass1_, TMBIR_N)(const GroupDev* gs, int n, const StepArgs& a, bool bf16, cudaStream_t s) {
  return pass1_n<TMBIR_N>(gs, n, a, bf16, s);
}
int TMBIR_CAT(pass2_, TMBIR_N)(const GroupDev* gs, int n, const IterState* st, bool bf16, cudaStream_t s) {
  return pass2_n<TMBIR_N>(gs, n, st, bf16, s);
}
int TMBIR_CAT(pass3_, TMBIR_N)(const GroupDev* gs, int n, const StepArgs& a, Pass3Mode m, const PriorC& pc,
                                double* partials, int off, bool bf16, int part, cudaStream_t s) {
  return pass3_n<TMBIR_N>(gs, n, a, m, pc, partials, off, bf16, part, s);
}
}  // namespace tmbir
