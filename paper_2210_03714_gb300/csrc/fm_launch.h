// fm_launch.h -- host-side entry points of the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "fm_job.h"

namespace fmk {

// dynamic shared memory of the persistent kernel for matrices up to dmax
size_t launch_smem(bool cplx, int nb, int dmax, bool tck = false);
// whether a (type, precision) pair runs the tensor-core kernel
inline bool uses_tc(bool cplx, int precision) { return !cplx && precision != 0; }
// resident CTAs per SM of the persistent kernel at that shared memory size
int launch_occupancy(bool cplx, int precision, int nb, size_t smem);
// the persistent kernel: grid CTAs, each pulling matrices from the queue
cudaError_t launch_persistent(bool cplx, int precision, int nb, const FmJob& J, const FmCoef& cf,
                              int grid, size_t smem, cudaStream_t st);
// order the batch by d (largest first), reset the queue, flag bad d in info;
// only orders in [lo, hi] enter the queue (a part of a split batch)
cudaError_t launch_order(const int* d, int batch, int dmax, int lo, int hi, int* order,
                         int* counter, int* info, cudaStream_t st);
// step a1 alone (fm_select_batched): s (steps = 0) or N (steps = 1) per matrix;
// fixed >= 0 (s) or > 0 (N) is written as given
cudaError_t launch_select(bool cplx, const int* d, const int64_t* off, const void* A,
                          const double* t, int batch, int dmax, double anorm, double theta,
                          int steps, long long fixed, long long* out, int* info, cudaStream_t st);
// autotuner probe matrices: hash-uniform entries in [-scale, scale)
cudaError_t launch_probe_fill(double* A, long long count, unsigned long long seed, double scale,
                              cudaStream_t st);
// per-type launchers (fm_inst_*.cu)
cudaError_t launch_real(int precision, int nb, const FmJob& J, const FmCoef& cf, int grid,
                        size_t smem, cudaStream_t st);
cudaError_t launch_cplx(int precision, int nb, const FmJob& J, const FmCoef& cf, int grid,
                        size_t smem, cudaStream_t st);
int occ_real(int precision, int nb, size_t smem);
int occ_cplx(int precision, int nb, size_t smem);

}  // namespace fmk
