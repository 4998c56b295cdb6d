// fm_launch.cu -- dispatch to the per-type kernels, and the batch-ordering kernel.
#include "fm_kernels.cuh"
#include "fm_launch.h"

namespace fmk {

size_t launch_smem(bool cplx, int nb, int dmax, bool tck) {
  if (cplx) return nb == 16 ? fm_smem_bytes<zd, 16>(dmax) : fm_smem_bytes<zd, 8>(dmax);
  return nb == 16 ? fm_smem_bytes<double, 16>(dmax, tck) : fm_smem_bytes<double, 8>(dmax, tck);
}

int launch_occupancy(bool cplx, int precision, int nb, size_t smem) {
  return cplx ? occ_cplx(precision, nb, smem) : occ_real(precision, nb, smem);
}

cudaError_t launch_persistent(bool cplx, int precision, int nb, const FmJob& J, const FmCoef& cf,
                              int grid, size_t smem, cudaStream_t st) {
  return cplx ? launch_cplx(precision, nb, J, cf, grid, smem, st)
              : launch_real(precision, nb, J, cf, grid, smem, st);
}

// Counting sort of the batch by d, largest first (longest jobs start first so
// the persistent CTAs finish together).  Matrices with d outside [1, dmax] get
// info = -4 and are left out of the queue.
__global__ void fm_order_kernel(const int* __restrict__ d, int batch, int dmax, int* order,
                                int* counter, int* info) {
  extern __shared__ int hist[];
  for (int i = threadIdx.x; i <= dmax; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    const int dd = d[b];
    if (dd >= 1 && dd <= dmax) atomicAdd(&hist[dmax - dd], 1);
    else if (info) info[b] = -4;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int i = 0; i <= dmax; ++i) {
      const int c = hist[i];
      hist[i] = run;
      run += c;
    }
    counter[0] = 0;
    counter[1] = run;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    const int dd = d[b];
    if (dd >= 1 && dd <= dmax) order[atomicAdd(&hist[dmax - dd], 1)] = b;
  }
}

cudaError_t launch_order(const int* d, int batch, int dmax, int* order, int* counter, int* info,
                         cudaStream_t st) {
  fm_order_kernel<<<1, 1024, (size_t)(dmax + 1) * sizeof(int), st>>>(d, batch, dmax, order,
                                                                       counter, info);
  return cudaGetLastError();
}

}  // namespace fmk
