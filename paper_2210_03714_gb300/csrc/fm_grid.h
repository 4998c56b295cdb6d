// fm_grid.h -- host side of the grid-wide path (one matrix over every SM),
// called by the C ABI for single-matrix calls of large order.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "fm_job.h"

namespace fmk {

struct GridJob {
  int kind;       // JOB_EXPM, JOB_PHI1, JOB_EXPMV or JOB_PHI1MV
  bool cplx;
  int precision;  // 0: products on the FP64 pipe; else tensor-core digit products
  int form;       // 0 roundoff, 1 plain
  int d, m;
  const void* A;
  int lda;
  double t;
  void* F;        // exp (or phi_1) result, ldf
  int ldf;
  void* E;        // phi_1 only: exp result (nullable), lde
  int lde;
  const void* V;  // actions: d x m, ldv
  int ldv;
  void* W;        // actions: d x m result, ldw
  int ldw;
  double anorm;
  int s_fixed;
  long long nsteps;
  int max_iters;  // limit of the correction iterations per shifted system
  FmCoef cf;
  void* ws;
  size_t ws_bytes;
  cudaStream_t st;
  int* info_host;
  int* s_host;
  long* n_host;
  void* stats;  // fm_stats of the calling thread (written during the call)
};

// CUDA events around each tensor-core tile launch of a call; their times are
// summed once the call has synchronized its stream
struct TileTimer {
  std::vector<cudaEvent_t> ev;  // start, stop pairs
  bool open = false;
  void start(cudaStream_t st) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    ev.push_back(a);
    ev.push_back(b);
    cudaEventRecord(a, st);
    open = true;
  }
  void stop(cudaStream_t st) {
    if (!open) return;
    cudaEventRecord(ev.back(), st);
    open = false;
  }
  double total_ms() const {  // after the stream is synchronized
    double t = 0;
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) t += ms;
    }
    return t;
  }
  ~TileTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

// scratch bytes the grid path needs
size_t grid_ws_bytes(int kind, bool cplx, int precision, int d, int m);

// runs the whole evaluation; returns an fm_status value and writes a message
// into msg on failure.  Synchronizes the stream (the step counts are chosen on
// the host from the norm computed on the device).
int grid_run(const GridJob& g, char* msg, size_t msglen);

}  // namespace fmk
