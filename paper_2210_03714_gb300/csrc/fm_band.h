// fm_band.h -- host side of the pentadiagonal action path (fm_band.cu), called
// by the C ABI for fm_band_expmv_batched with half bandwidth 2.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "fm_job.h"

namespace fmk {

struct PentaJob {
  int batch, d;
  int form;              // 0 roundoff (Eq. ParallRoundOff), 1 plain (Eq. rat1)
  const double* diags;   // 5 diagonals: A[k][k + o] of system b at ((o + 2) d + k) batch + b
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
size_t penta_ws_bytes(int batch, int d, int k);

// launches the factorization and the N steps (stream-ordered, no host
// synchronization); returns an fm_status value
int penta_run(const PentaJob& j, char* msg, size_t len);

}  // namespace fmk
