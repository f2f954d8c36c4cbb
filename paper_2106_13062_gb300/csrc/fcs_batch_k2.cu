// fcs_batch_k2.cu -- batch class kernels for FFT length P = 8192
// (log2 M = 12), both thread multipliers.
#include "fcs_batch_kernels.cuh"

namespace fcs {

ClassKernel class_kernel_12(int ntm, int ipc, int64_t Imax, int sb) {
  return class_kernel_l<12>(ntm, ipc, Imax, sb);
}

}  // namespace fcs
