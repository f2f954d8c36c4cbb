// fcs_batch_k4.cu -- batch class kernels for FFT lengths P = 256 .. 1024
// (log2 M = 7 .. 9), both thread multipliers.
#include "fcs_batch_kernels.cuh"

namespace fcs {

ClassKernel class_kernel_small2(int L, int ntm, int ipc, int64_t Imax, int sb) {
  switch (L) {
#define FCS_CLASS_CASE(K) \
  case K: return class_kernel_l<K>(ntm, ipc, Imax, sb);
    FCS_CLASS_CASE(7) FCS_CLASS_CASE(8) FCS_CLASS_CASE(9)
#undef FCS_CLASS_CASE
    default:
      return ClassKernel{nullptr, 0, 0};
  }
}

}  // namespace fcs
