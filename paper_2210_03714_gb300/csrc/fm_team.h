// fm_team.h -- host side of the team path: one matrix of small order, every
// step spread over many SMs in one cooperative launch (fm_team.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "fm_job.h"

namespace fmk {

struct TeamJob {
  bool cplx;
  int form;
  int n;
  const void* A;
  int lda;
  double t;
  void* F;
  int ldf;
  double anorm;
  int s_fixed;
  FmCoef cf;
  void* ws;
  size_t ws_bytes;
  cudaStream_t st;
  int* info_host;  // nullable; written after the stream is synchronized
  int* s_host;     // nullable
};

// largest order the team path takes
constexpr int kTeamMaxDim = 512;

// shifted systems of a set (the +-c pairs of the roundoff form fused)
int team_systems(const FmCoef& cf, int form);

// device scratch for one call of order n with nsys shifted systems
size_t team_ws_bytes(bool cplx, int n, int nsys);

// runs exp(tA) of the job (synchronizes its stream to read the status);
// FM_* status, message in msg
int team_run(const TeamJob& j, char* msg, size_t len);

}  // namespace fmk
