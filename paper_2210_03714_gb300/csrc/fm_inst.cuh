// fm_inst.cuh -- instantiation helper for one (working type, factor type) pair.
#pragma once
#include "fm_kernels.cuh"
#include "fm_launch.h"

namespace fmk {

template <class T, class TL>
using KernelPtr = void (*)(FmJob, FmCoef);

template <class T, class TL, bool TCK>
KernelPtr<T, TL> pick_kernel(int nb) {
  return nb == 16 ? fm_persistent<T, TL, 16, TCK> : fm_persistent<T, TL, 8, TCK>;
}

template <class T, class TL, bool TCK = false>
cudaError_t launch_pair(int nb, const FmJob& J, const FmCoef& cf, int grid, size_t smem,
                        cudaStream_t st) {
  KernelPtr<T, TL> k = pick_kernel<T, TL, TCK>(nb);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, NT, smem, st>>>(J, cf);
  return cudaGetLastError();
}

template <class T, class TL, bool TCK = false>
int occ_pair(int nb, size_t smem) {
  KernelPtr<T, TL> k = pick_kernel<T, TL, TCK>(nb);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n;
}

}  // namespace fmk
