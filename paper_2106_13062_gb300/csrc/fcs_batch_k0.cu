// fcs_batch_k0.cu -- batch class kernels for FFT lengths P = 16 .. 128
// (log2 M = 3 .. 6), both thread multipliers.
#include "fcs_batch_kernels.cuh"

namespace fcs {

ClassKernel class_kernel_small(int L, int ntm, int ipc, int64_t Imax, int sb) {
  switch (L) {
#define FCS_CLASS_CASE(K) \
  case K: return class_kernel_l<K>(ntm, ipc, Imax, sb);
    FCS_CLASS_CASE(3) FCS_CLASS_CASE(4) FCS_CLASS_CASE(5) FCS_CLASS_CASE(6)
#undef FCS_CLASS_CASE
    default:
      return class_kernel_small2(L, ntm, ipc, Imax, sb);
  }
}

}  // namespace fcs
