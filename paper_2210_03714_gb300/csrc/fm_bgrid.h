// fm_bgrid.h -- host side of the grid path over a batch of matrices (exp),
// called by the C ABI for batched calls on FM_PATH_GRID.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fm_job.h"

namespace fmk {

struct BGridJob {
  int kind;                // JOB_EXPM, JOB_PHI1 or JOB_PHI1MV
  bool cplx;
  int form;
  int batch;
  const int* d_host;       // orders (host copy)
  const int64_t* off_host; // element offsets of the caller's matrices (host copy)
  const void* A;           // packed input (device)
  const double* t_dev;
  void* F;                 // packed output (device, same offsets): exp or phi_1
  void* E;                 // phi_1: exp output (nullable), same offsets
  const void* V;           // phi_1 action: V_b (d_b x m) at voff_host[b]
  void* W;                 // phi_1 action: W_b = phi_1(t_b A_b) V_b, same offsets
  const int64_t* voff_host;
  int m;
  int* info_dev;
  int* s_dev;              // nullable
  double anorm;
  int s_fixed;
  int max_iters;
  FmCoef cf;
  void* ws;
  size_t ws_bytes;
  cudaStream_t st;
  void* stats;             // fm_stats of the calling thread
};

// scratch bytes for a batch of these orders
size_t bgrid_ws_bytes(int kind, bool cplx, int batch, const int* d_host);

// runs exp(t_b A_b) (or phi_1, or phi_1 times V) for the whole batch;
// synchronizes the stream (the step counts are read back between launches).
// Returns an fm_status value.
int bgrid_run(const BGridJob& j, char* msg, size_t len);

}  // namespace fmk
