// Kernels for real matrices: double everywhere, or single-precision factors.
#include "fm_inst.cuh"

namespace fmk {

cudaError_t launch_real(int precision, int nb, const FmJob& J, const FmCoef& cf, int grid,
                        size_t smem, cudaStream_t st) {
  if (precision == 0) return launch_pair<double, double>(nb, J, cf, grid, smem, st);
  // mixed precision: single-precision factors, double-accurate products on the
  // tensor cores
  return launch_pair<double, float, true>(nb, J, cf, grid, smem, st);
}

int occ_real(int precision, int nb, size_t smem) {
  return precision == 0 ? occ_pair<double, double>(nb, smem)
                        : occ_pair<double, float, true>(nb, smem);
}

}  // namespace fmk
