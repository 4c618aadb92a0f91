// Definitions of the patch-kernel launchers, instantiated for one degree
// (both precisions) by each patch_k<K>.cu.
#pragma once

#include <algorithm>

#include "patch_kernel.cuh"

namespace stk {

template <int K, typename T>
cudaError_t launch_patch_k(PatchArgs<T> a, int nblocks, cudaStream_t s) {
  using C = PatchThreads<K, T>;
  const size_t smem = patch_smem_bytes<K>(sizeof(T));
  static std::atomic<unsigned long long> smem_set{0}, smem_set_interior{0}, smem_set_f{0}, smem_set_fi{0};
  const bool fused = a.mode == 3;
  {
    cudaError_t e = fused ? allow_dynamic_smem(patch_kernel<K, T, true>, smem, smem_set_f)
                          : allow_dynamic_smem(patch_kernel<K, T>, smem, smem_set);
    if (e == cudaSuccess)
      e = fused ? allow_dynamic_smem(patch_kernel_interior<K, T, true>, smem, smem_set_fi)
                : allow_dynamic_smem(patch_kernel_interior<K, T>, smem, smem_set_interior);
    if (e != cudaSuccess) return e;
  }
  if (nblocks > 0) {
    const bool interior = (a.mode == 0 || fused) && a.part == 1;
    InteriorMats<K, T> im{};  // read by the FP32 interior kernel only
    if constexpr (sizeof(T) == 4) {
      if (interior) {
        if (!a.htab) return cudaErrorInvalidValue;
        constexpr int NE = InteriorMats<K, T>::NE;
        std::copy(a.htab->SC, a.htab->SC + NE, im.SC);
        std::copy(a.htab->SD[0], a.htab->SD[0] + NE, im.SD);
        std::copy(a.htab->EC, a.htab->EC + NE, im.EC);
        std::copy(a.htab->FM[0], a.htab->FM[0] + NE, im.FM);
      }
    }
    if (fused) {
      if (interior)
        patch_kernel_interior<K, T, true><<<nblocks, C::NT, smem, s>>>(a, im);
      else
        patch_kernel<K, T, true><<<nblocks, C::NT, smem, s>>>(a);
    } else if (interior) {
      patch_kernel_interior<K, T><<<nblocks, C::NT, smem, s>>>(a, im);
    } else {
      patch_kernel<K, T><<<nblocks, C::NT, smem, s>>>(a);
    }
  }
  return cudaGetLastError();
}

template <int K, typename T>
cudaError_t launch_patch_multi_k(const PatchArgs<T>& a, const PatchJobs<T>& J, int nblocks, cudaStream_t s) {
  using C = PatchThreads<K, T>;
  const size_t smem = patch_smem_bytes<K>(sizeof(T));
  static std::atomic<unsigned long long> smem_set{0};
  {
    const cudaError_t e = allow_dynamic_smem(patch_kernel_multi<K, T>, smem, smem_set);
    if (e != cudaSuccess) return e;
  }
  if (nblocks > 0) patch_kernel_multi<K, T><<<nblocks, C::NT, smem, s>>>(a, J);
  return cudaGetLastError();
}

#define STK_PATCH_INSTANTIATE(KK)                                                                       \
  template cudaError_t launch_patch_k<KK, float>(PatchArgs<float>, int, cudaStream_t);                  \
  template cudaError_t launch_patch_k<KK, double>(PatchArgs<double>, int, cudaStream_t);                \
  template cudaError_t launch_patch_multi_k<KK, float>(const PatchArgs<float>&, const PatchJobs<float>&, \
                                                       int, cudaStream_t);                              \
  template cudaError_t launch_patch_multi_k<KK, double>(const PatchArgs<double>&,                      \
                                                        const PatchJobs<double>&, int, cudaStream_t);

}  // namespace stk
