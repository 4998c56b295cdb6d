// fm_job.h -- launch descriptors shared by the host API and the kernels.
#pragma once
#include <stddef.h>
#include <stdint.h>

#ifdef __CUDACC__
#define FM_HD __host__ __device__ __forceinline__
#else
#define FM_HD inline
#endif

namespace fmk {

constexpr int kMaxTerms = 16;

// Coefficients of one or two functions sharing the nodes c_i (Sec. 2: the
// same resolvents serve several functions through different weights).
struct FmCoef {
  int k;          // number of terms
  int nfun;       // 1 (exp) or 2 (exp, phi_1)
  int conj_pair;  // unused by the kernels (rejected on the host for now)
  int pad;
  double c_re[kMaxTerms], c_im[kMaxTerms];
  double b_re[2][kMaxTerms], b_im[2][kMaxTerms];
  double a0[2], d1[2], d2[2];
  double theta;   // min over the functions
};

enum { JOB_EXPM = 0, JOB_PHI1 = 1, JOB_EXPMV = 2, JOB_PHI1MV = 3, JOB_ADJ = 4 };

struct FmJob {
  int kind, precision, form, max_ir;
  double ir_tol, anorm;
  int s_fixed;
  int batch, dmax, m;
  long long nsteps;       // > 0: forced step count (actions)
  long long nsteps_max;   // adjoint: workspace bound on N
  // batched mode: d/off/voff are device arrays; single mode: d == nullptr
  const int* d;
  const int64_t* off;
  const int64_t* voff;
  int d1, lda, ldf, lde, ldv, ldw;
  const double* t;
  double t1;
  const void* A;
  void* F;
  void* E;
  const void* V;
  void* W;
  int* info;
  int* sN;
  const long long* nsteps_dev;  // adjoint
  const double* wbar;
  double* Abar;
  double* vbar;
  char* ws;
  size_t ws_stride;  // bytes of scratch per CTA
  const int* order;  // matrices sorted by d, largest first
  int* counter;      // work queue head
  size_t smem_avail; // bytes of shared memory the per-matrix routines may use
};

FM_HD size_t fm_align(size_t x) { return (x + 255) & ~(size_t)255; }

// Per-CTA scratch layout.  elt = sizeof of the working type T, lelt = sizeof
// of the factorization type TL.  Offsets are computed identically on the host
// (to size the buffer) and on the device (to carve it).
struct WsLayout {
  size_t B, C, Y, F, Phi, T1, T2, B2, LU, RL, piv, D;  // matrix-function part
  size_t Cs, LUs, pivs, Ds, Wc, Wn, U, U2, RHS;    // action part
  size_t Wst, Yst, Lam, Yt;                        // adjoint part
  size_t gx, gy, ex, fy;                           // digit planes (tensor-core products)
  size_t total;
};

// digit-plane bytes of the tensor-core products (see ozaki.cuh): X operands up
// to n x n, Y operands up to n x max(n, m); tiles of 128 x 32 and 64 x 32
FM_HD size_t oz_x_bytes(int n) { return (size_t)((n + 127) / 128) * ((n + 31) / 32) * (7 * 128 * 32 * 2); }
FM_HD size_t oz_y_bytes(int n, int m) {
  int w = n > m ? n : m;
  return (size_t)((w + 63) / 64) * ((n + 31) / 32) * (7 * 64 * 32 * 2);
}

FM_HD WsLayout ws_layout(int kind, int n, int m, int k, size_t elt, size_t lelt,
                         long long nmax, int tc = 0) {
  WsLayout L = {};
  size_t o = 0;
  const size_t nn = (size_t)n * n;
  const size_t nm = (size_t)n * (m > 0 ? m : 1);
  auto take = [&](size_t bytes) { size_t r = o; o += fm_align(bytes); return r; };
  const size_t big = nn > nm ? nn : nm;
  L.B = take(nn * elt);
  L.C = take(nn * elt);
  L.Y = take(big * elt);
  L.T1 = take(big * elt);
  L.RL = take(big * lelt);
  L.D = take((size_t)n * 8 * 2);
  if (kind == JOB_EXPM || kind == JOB_PHI1 || kind == JOB_PHI1MV) {
    L.F = take(nn * elt);
    L.Phi = take(nn * elt);
    L.T2 = take(nn * elt);
    L.B2 = take(nn * elt);
    L.LU = take(nn * lelt);
    L.piv = take((size_t)n * 4);
  } else {
    L.Cs = take((size_t)k * nn * elt);
    L.LUs = take((size_t)k * nn * lelt);
    L.pivs = take((size_t)k * n * 4);
    L.Ds = take((size_t)k * n * 8 * 2);
    L.Wc = take(nm * elt);
    L.Wn = take(nm * elt);
    L.U = take(nm * elt);
    L.U2 = take(nm * elt);
    L.RHS = take(nm * elt);
    if (kind == JOB_ADJ) {
      L.Wst = take((size_t)(nmax + 1) * n * elt);
      L.Yst = take((size_t)nmax * k * n * elt);
      L.Lam = take((size_t)n * (k + 1) * elt);
      L.Yt = take((size_t)n * (k + 1) * elt);
    }
  }
  if (tc) {
    const int w = n > m ? n : m;
    L.gx = take(oz_x_bytes(n));
    L.gy = take(oz_y_bytes(n, m));
    L.ex = take((size_t)((n + 127) / 128) * 128 * 4);
    L.fy = take((size_t)((w + 63) / 64) * 64 * 4);
  }
  L.total = o;
  return L;
}

}  // namespace fmk
