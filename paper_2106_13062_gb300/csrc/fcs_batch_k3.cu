// fcs_batch_k3.cu -- batch class kernels for FFT length P = 16384 on the
// warp-DIT engine (512 threads; prefetch depth from the longest mode and
// scatter-buffer height from the longest hash range).
#include "fcs_batch_kernels.cuh"

namespace fcs {
namespace {

template <int CPT, bool MULTI>
const void *class13_fn(int ra) {
  if (ra <= 128) return reinterpret_cast<const void *>(batch_class13_kernel<CPT, 4, MULTI>);
  if (ra <= 256) return reinterpret_cast<const void *>(batch_class13_kernel<CPT, 8, MULTI>);
  return reinterpret_cast<const void *>(batch_class13_kernel<CPT, 16, MULTI>);
}
template <bool MULTI>
const void *class13_pick(int cpt, int ra) {
  return cpt <= 1 ? class13_fn<1, MULTI>(ra) : cpt <= 2 ? class13_fn<2, MULTI>(ra)
                                                        : class13_fn<4, MULTI>(ra);
}

}  // namespace

ClassKernel class_kernel_13(int ipc, int64_t Imax, int sb) {
  const int ra = (sb + 31) >> 5;
  const int cpt = int((Imax + wdit::kNT - 1) / wdit::kNT);
  const void *fn = ipc > 1 ? class13_pick<true>(cpt, ra) : class13_pick<false>(cpt, ra);
  return ClassKernel{fn, wdit::kNT, Cp13Smem::bytes(ra)};
}

}  // namespace fcs
