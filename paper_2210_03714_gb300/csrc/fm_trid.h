// fm_trid.h -- host side of the tridiagonal action path (fm_trid.cu), called
// by the C ABI for fm_trid_expmv_batched.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "fm_job.h"

namespace fmk {

struct TridJob {
  int batch, d;
  int form;              // 0 roundoff (Eq. ParallRoundOff), 1 plain (Eq. rat1)
  const double* dl;      // sub-diagonal, element k of system b at k * batch + b (k >= 1)
  const double* dd;      // diagonal
  const double* du;      // super-diagonal (k <= d - 2)
  const double* t;       // device, batch times
  const double* V;       // device, batch-interleaved vectors
  double* W;             // device, batch-interleaved results
  int* info;             // device, batch
  int* nsteps;           // device, batch (nullable)
  double anorm;          // > 0: anorm |t_b| replaces ||t_b A_b||_1
  long nsteps_fixed;     // > 0: N for every system
  FmCoef cf;
  void* ws;
  size_t ws_bytes;
  cudaStream_t st;
};

// scratch bytes for a batch of systems of order d with k terms
size_t trid_ws_bytes(int batch, int d, int k);

// launches the factorization and the N steps (stream-ordered, no host
// synchronization); returns an fm_status value
int trid_run(const TridJob& j, char* msg, size_t len);

}  // namespace fmk
