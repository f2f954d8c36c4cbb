// fcs_batch_k2.cu -- batch class kernels for FFT length P = 8192
// (log2 M = 12): the slot FFT at both thread multipliers, and the warp-DIT
// engine (256 threads, two CTAs per SM).
#include "fcs_batch_kernels.cuh"

namespace fcs {
namespace {

template <int CPT, bool MULTI>
const void *class12w_fn(int ra) {
  if (ra <= 128) return reinterpret_cast<const void *>(batch_class12w_kernel<CPT, 4, MULTI>);
  if (ra <= 256) return reinterpret_cast<const void *>(batch_class12w_kernel<CPT, 8, MULTI>);
  return reinterpret_cast<const void *>(batch_class12w_kernel<CPT, 16, MULTI>);
}
template <bool MULTI>
const void *class12w_pick(int cpt, int ra) {
  return cpt <= 1 ? class12w_fn<1, MULTI>(ra) : cpt <= 2 ? class12w_fn<2, MULTI>(ra)
                                                         : class12w_fn<4, MULTI>(ra);
}

}  // namespace

ClassKernel class_kernel_12(int eng, int ntm, int ipc, int64_t Imax, int sb) {
  if (eng == 1) {
    const int ra = (sb + 15) >> 4;
    const int cpt = int((Imax + wdit::w12::kNT - 1) / wdit::w12::kNT);
    const void *fn = ipc > 1 ? class12w_pick<true>(cpt, ra) : class12w_pick<false>(cpt, ra);
    return ClassKernel{fn, wdit::w12::kNT, Cp12Smem::bytes(ra)};
  }
  return class_kernel_l<12>(ntm, ipc, Imax, sb);
}

}  // namespace fcs
