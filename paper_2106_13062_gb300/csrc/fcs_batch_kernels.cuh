// fcs_batch_kernels.cuh -- the per-FFT-size class kernels of a batch plan
// (eq. FCS_syn over many CP problems) and the host-side picker of one class
// kernel for a tuned configuration.  The kernels are instantiated in several
// translation units (fcs_batch_k*.cu, one range of FFT sizes each) so that
// the variants compile in parallel.  Not part of the ABI.
#pragma once

#include "fcs_batch_internal.cuh"
#include "fcs_cp_run.cuh"

namespace fcs {

// Problem descriptor in device memory (one per problem of a plan).
struct BatchProb {
  int N, D, L, sb;
  int64_t R, rpi;
  int64_t I[kMaxN], off[kMaxN], ut_off[kMaxN];
  int64_t ldh, Jt;
  const float *UT;
  const int32_t *h;
  const int8_t *s;
  float2 *G;
  unsigned *tickets;
  float *out;
  int groups;
  int pad_;
};

// cp_run / cp13_run's accessors over a problem descriptor (fcs_cp_run.cuh).
struct BatchView {
  const BatchProb &P;
  int sb;
  // factor columns and tables, written before the chain's first class
  template <class T>
  __device__ __forceinline__ T ld(const T *p) const {
    return __ldg(p);
  }
  __device__ __forceinline__ int modes() const { return P.N; }
  __device__ __forceinline__ int64_t dim(int n) const { return P.I[n]; }
  __device__ __forceinline__ const float *column(int n, int64_t r) const {
    return P.UT + P.ut_off[n] + r * P.I[n];
  }
  __device__ __forceinline__ const int32_t *hashes(int d, int n) const {
    return P.h + d * P.ldh + P.off[n];
  }
  __device__ __forceinline__ const int8_t *signs(int d, int n) const {
    return P.s + d * P.ldh + P.off[n];
  }
  __device__ __forceinline__ int64_t length() const { return P.Jt; }
  __device__ __forceinline__ float *sketch(int d) const { return P.out + d * P.Jt; }
  __device__ __forceinline__ float2 *spectrum() const { return P.G; }
  __device__ __forceinline__ unsigned *ticket(int d) const { return P.tickets + d; }
};

// Kernel, block size and shared memory of one class configuration.
struct ClassKernel {
  const void *fn;
  int nt;
  size_t smem;
};

// Threads of the slot FFT for log2 M = L at thread multiplier ntm (1: one
// radix-16 butterfly per thread, at least a warp; 2: twice that, at most 1024).
__host__ __device__ constexpr int class_threads(int L, int ntm) {
  return fft_threads(L) * ntm > 1024 ? 1024 : fft_threads(L) * ntm;
}

// Per-range pickers, one translation unit each (null fn outside the range).
ClassKernel class_kernel_small(int L, int ntm, int ipc, int64_t Imax, int sb);  // L = 3 .. 9
ClassKernel class_kernel_small2(int L, int ntm, int ipc, int64_t Imax, int sb); // L = 7 .. 9
ClassKernel class_kernel_mid(int L, int ntm, int ipc, int64_t Imax, int sb);    // L = 10, 11
ClassKernel class_kernel_12(int eng, int ntm, int ipc, int64_t Imax, int sb);   // L = 12
ClassKernel class_kernel_13(int ipc, int64_t Imax, int sb);                     // L = 13

// The kernels have internal linkage: each translation unit instantiates only
// its own range of FFT sizes.
namespace {

// Programmatic dependent launch.  launch_dependents lets the next launch of
// the chain start once every CTA of this grid has issued it (so every CTA of
// this grid is already resident: the next grid can never hold the SMs this
// one still needs).  wait_previous returns once the previous grid of the
// chain has completed and its writes are visible; called at a CTA's end, it
// makes each grid complete after its predecessor, so work queued after the
// chain waits for all of it.  Both are no-ops in a launch made without the
// programmatic-serialisation attribute.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_previous() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// One work item (problem, sketch d, rank group) of an FFT-size class per CTA
// (MULTI = false), or the items [ipc * blockIdx.x, ...), at most ipc of them,
// one after another (MULTI = true; a separate instantiation so that the
// one-item kernel keeps its register allocation).  P = 2^(LOG2M+1) <= 8192
// on NT threads.
template <int LOG2M, int NT, int CPT, bool MULTI>
__global__ void __launch_bounds__(NT) batch_class_kernel(const BatchProb *__restrict__ probs,
                                                         const int4 *__restrict__ items,
                                                         const float2 *__restrict__ tw,
                                                         int count, int ipc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int is_last;
  pdl_launch_dependents();
  auto one = [&](int it) {
    const int4 w = items[it];
    const BatchProb &P = probs[w.x];
    const int64_t r0 = int64_t(w.z) * P.rpi;
    const int64_t r1 = min(P.R, r0 + P.rpi);
    const BatchView view{P, P.sb};
    cp_run<LOG2M, NT, CPT>(view, w.y, r0, r1, unsigned(P.groups), smem_raw, tw, &is_last);
  };
  if constexpr (MULTI) {
    const int first = blockIdx.x * ipc, last = min(count, first + ipc);
    for (int it = first; it < last; ++it) {
      if (it > first) __syncthreads();       // shared memory of the previous item
      one(it);
    }
  } else {
    one(blockIdx.x);
  }
  pdl_wait_previous();
}

// The same for P = 16384 on the warp-DIT engine (ra <= 32 RMAX).
template <int CPT, int RMAX, bool MULTI>
__global__ void __launch_bounds__(wdit::kNT) batch_class13_kernel(
    const BatchProb *__restrict__ probs, const int4 *__restrict__ items,
    const float2 *__restrict__ tw, int count, int ipc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int is_last;
  pdl_launch_dependents();
  auto one = [&](int it) {
    const int4 w = items[it];
    const BatchProb &P = probs[w.x];
    const int64_t r0 = int64_t(w.z) * P.rpi;
    const int64_t r1 = min(P.R, r0 + P.rpi);
    const BatchView view{P, P.sb};
    cp13_run<CPT, RMAX>(view, w.y, r0, r1, unsigned(P.groups), smem_raw, tw, &is_last);
  };
  if constexpr (MULTI) {
    const int first = blockIdx.x * ipc, last = min(count, first + ipc);
    for (int it = first; it < last; ++it) {
      if (it > first) __syncthreads();
      one(it);
    }
  } else {
    one(blockIdx.x);
  }
  pdl_wait_previous();
}

// The same for P = 8192 on the warp-DIT engine of wdit::w12 (256 threads,
// two CTAs per SM; ra <= 32 RMAX).
template <int CPT, int RMAX, bool MULTI>
__global__ void __launch_bounds__(wdit::w12::kNT, 2) batch_class12w_kernel(
    const BatchProb *__restrict__ probs, const int4 *__restrict__ items,
    const float2 *__restrict__ tw, int count, int ipc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int is_last;
  pdl_launch_dependents();
  auto one = [&](int it) {
    const int4 w = items[it];
    const BatchProb &P = probs[w.x];
    const int64_t r0 = int64_t(w.z) * P.rpi;
    const int64_t r1 = min(P.R, r0 + P.rpi);
    const BatchView view{P, P.sb};
    cp12_run<CPT, RMAX>(view, w.y, r0, r1, unsigned(P.groups), smem_raw, tw, &is_last);
  };
  if constexpr (MULTI) {
    const int first = blockIdx.x * ipc, last = min(count, first + ipc);
    for (int it = first; it < last; ++it) {
      if (it > first) __syncthreads();
      one(it);
    }
  } else {
    one(blockIdx.x);
  }
  pdl_wait_previous();
}

// Slot-FFT class kernel for log2 M = L with NT threads: prefetch depth from
// the class's longest mode (entries per thread, the rest scattered directly).
template <int L, int NT, bool MULTI>
ClassKernel class_kernel_nt(int64_t Imax, int sb) {
  const int cpt = int((Imax + NT - 1) / NT);
  ClassKernel k{nullptr, NT, CpSmem<L, NT>::bytes(sb)};
  if (cpt <= 1)
    k.fn = reinterpret_cast<const void *>(batch_class_kernel<L, NT, 1, MULTI>);
  else if (cpt <= 2)
    k.fn = reinterpret_cast<const void *>(batch_class_kernel<L, NT, 2, MULTI>);
  else
    k.fn = reinterpret_cast<const void *>(batch_class_kernel<L, NT, 4, MULTI>);
  return k;
}

template <int L>
ClassKernel class_kernel_l(int ntm, int ipc, int64_t Imax, int sb) {
  if (ntm == 2)
    return ipc > 1 ? class_kernel_nt<L, class_threads(L, 2), true>(Imax, sb)
                   : class_kernel_nt<L, class_threads(L, 2), false>(Imax, sb);
  return ipc > 1 ? class_kernel_nt<L, class_threads(L, 1), true>(Imax, sb)
                 : class_kernel_nt<L, class_threads(L, 1), false>(Imax, sb);
}

}  // namespace
}  // namespace fcs
