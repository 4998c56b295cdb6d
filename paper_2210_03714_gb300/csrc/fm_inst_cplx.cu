// Kernels for complex matrices: complex double, or complex single factors.
#include "fm_inst.cuh"

namespace fmk {

cudaError_t launch_cplx(int precision, int nb, const FmJob& J, const FmCoef& cf, int grid,
                        size_t smem, cudaStream_t st) {
  if (precision == 0) return launch_pair<zd, zd>(nb, J, cf, grid, smem, st);
  return launch_pair<zd, zf>(nb, J, cf, grid, smem, st);
}

int occ_cplx(int precision, int nb, size_t smem) {
  return precision == 0 ? occ_pair<zd, zd>(nb, smem) : occ_pair<zd, zf>(nb, smem);
}

}  // namespace fmk
