// fcs_batch_k1.cu -- batch class kernels for FFT lengths P = 2048 and 4096
// (log2 M = 10, 11), both thread multipliers.
#include "fcs_batch_kernels.cuh"

namespace fcs {

ClassKernel class_kernel_mid(int L, int ntm, int ipc, int64_t Imax, int sb) {
  if (L == 10) return class_kernel_l<10>(ntm, ipc, Imax, sb);
  if (L == 11) return class_kernel_l<11>(ntm, ipc, Imax, sb);
  return ClassKernel{nullptr, 0, 0};
}

}  // namespace fcs
