// fm_trid.cu -- exp(t_b A_b) v_b for a batch of tridiagonal A_b.  Sec. 2.1
// (functions of tridiagonal matrices acting on vectors) and Sec. 5: every
// shifted matrix I - c_i B of a tridiagonal B is tridiagonal, so its system is
// solved by the Thomas algorithm, 8d flops in the plain form (Eq. rat1) and,
// with the product B v, 13d in the roundoff form (Eq. ParallRoundOff; the
// paper's R'_10).  The steps are the action recurrence of Sec. 1: N steps
// v <- r(B) v with B = (t/N) A.
//
// One thread per system, the batch interleaved (element k of system b at
// k * batch + b), so a warp's loads at one k are contiguous.  Two launches:
//   trid_prep   finiteness; eta = ||t A||_1 (column sums in row order, as the
//               dense path forms them); N = max(1, ceil(eta / theta));
//               h = t / N; and the factors of every I - c_i h A, once for all
//               N steps.  With m, l, u the diagonal, sub- and super-diagonal
//               of I - c_i B:  beta_0 = m_0, lam_k = l_k / beta_{k-1},
//               beta_k = m_k - lam_k u_{k-1}; stored: lam_k, 1/beta_k and
//               g_k = u_k / beta_k (one division per node and row: the
//               quotients are products with 1/beta).  No pivoting: |c_i| ||B||_1 is far below
//               1/2 for the sets here at ||B||_1 <= theta, so I - c_i B is
//               diagonally dominant.  An exactly zero pivot stops the system
//               with info = i d + (1-based row), i the first such term.
//   trid_steps  the N steps.  Forward sweep over k for all nodes at once,
//               z_i,k = rhs_k - lam_i,k z_i,k-1 (rhs = B v in the roundoff
//               form, v in the plain form), z kept in scratch, and the base
//               a0' v + d1 B v + d2 B^2 v written to the step's output;
//               backward sweep y_i,k = z_i,k / beta_i,k - g_i,k y_i,k+1 and
//               w_k = base_k + sum_i w_i y_i,k (w_i = b_i c_i, or b_i).
// Per node and element a step costs 4 FP64 operations and 40 bytes (three
// factor reads, z written and read back).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/fm.h"
#include "fm_trid.h"

namespace fmk {
namespace {

constexpr int kThreads = 128;
// one warp per block for the steps: the FP64 pipe of each SM is their limit,
// and single-warp blocks spread the systems evenly over the SMs
constexpr int kStepThreads = 32;

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

// scratch: N and h per system, then lam, 1/beta, g and z ([node][k][b]) and
// the second step vector
struct TLay {
  size_t ns, h, lam, ib, g, z, sv, total;
};
TLay tlay(int batch, int d, int k) {
  TLay L;
  size_t o = 0;
  const size_t per = (size_t)k * d * batch * 8;
  L.ns = o; o += up((size_t)batch * 4);
  L.h = o; o += up((size_t)batch * 8);
  L.lam = o; o += up(per);
  L.ib = o; o += up(per);
  L.g = o; o += up(per);
  L.z = o; o += up(per);
  L.sv = o; o += up((size_t)d * batch * 8);
  L.total = o;
  return L;
}

struct TArgs {
  int batch, n, kn, roundoff, need_bv, need_b2;
  const double *dl, *dd, *du, *t, *V;
  double* W;
  int* info;
  int* nsteps;
  double anorm;
  long long nsteps_fixed;
  double theta, a0p, d1, d2;
  double c[kMaxTerms], w[kMaxTerms];  // nonzero nodes and their weights
  int idx[kMaxTerms];                 // their index in the coefficient set
  int* ns;
  double* h;
  double *lam, *ib, *g, *z, *sv;
};

// finiteness, N, h and the factors; one thread per system
__global__ void trid_prep(TArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.batch) return;
  const int n = a.n;
  const size_t S = a.batch;
  const double t = a.t[b];
  bool bad = !isfinite(t);
  double eta = 0.0;
  for (int k = 0; k < n; ++k) {
    // column k of t A: rows k-1, k, k+1
    const double up_ = k > 0 ? a.du[(size_t)(k - 1) * S + b] : 0.0;
    const double dk = a.dd[(size_t)k * S + b];
    const double lo = k + 1 < n ? a.dl[(size_t)(k + 1) * S + b] : 0.0;
    bad |= !isfinite(up_) || !isfinite(dk) || !isfinite(lo) || !isfinite(a.V[(size_t)k * S + b]);
    double s = __dadd_rn(fabs(__dmul_rn(t, up_)), fabs(__dmul_rn(t, dk)));
    s = __dadd_rn(s, fabs(__dmul_rn(t, lo)));
    eta = (s > eta || isnan(s)) ? s : eta;
  }
  if (bad) {
    a.info[b] = -2;
    a.ns[b] = 0;
    if (a.nsteps) a.nsteps[b] = 0;
    return;
  }
  if (a.anorm > 0) eta = __dmul_rn(a.anorm, fabs(t));
  long long N = a.nsteps_fixed;
  if (N <= 0) {
    const double q = ceil(eta / a.theta);
    N = q < 1.0 ? 1 : (q > 2147483647.0 ? 2147483647LL : (long long)q);
  }
  const double h = t / (double)N;
  // factors, k outer so the diagonals are read once; 1/beta and u of the
  // previous row per node (local arrays: this runs once per call)
  double beta[kMaxTerms], uprev[kMaxTerms];
  int zrow[kMaxTerms];
  for (int j = 0; j < a.kn; ++j) zrow[j] = 0;
  for (int k = 0; k < n; ++k) {
    const double hdd = __dmul_rn(h, a.dd[(size_t)k * S + b]);
    const double hdl = k > 0 ? __dmul_rn(h, a.dl[(size_t)k * S + b]) : 0.0;
    const double hdu = k + 1 < n ? __dmul_rn(h, a.du[(size_t)k * S + b]) : 0.0;
    for (int j = 0; j < a.kn; ++j) {
      const double c = a.c[j];
      const double m = __dsub_rn(1.0, __dmul_rn(c, hdd));
      const size_t at = ((size_t)j * n + k) * S + b;
      double bet = m;
      if (k > 0) {
        const double l = -__dmul_rn(c, hdl);
        const double lam = __dmul_rn(l, beta[j]);  // beta[j] holds 1 / beta_{k-1}
        bet = __dsub_rn(m, __dmul_rn(lam, uprev[j]));
        a.lam[at] = lam;
      }
      if (bet == 0.0 && zrow[j] == 0) zrow[j] = k + 1;
      const double u = k + 1 < n ? -__dmul_rn(c, hdu) : 0.0;
      const double r = 1.0 / bet;  // the one division per node and row
      a.ib[at] = r;
      a.g[at] = __dmul_rn(u, r);
      beta[j] = r;
      uprev[j] = u;
    }
  }
  int info = 0;
  for (int j = 0; j < a.kn && !info; ++j)
    if (zrow[j]) info = a.idx[j] * n + zrow[j];
  a.info[b] = info;
  a.ns[b] = info ? 0 : (int)N;
  a.h[b] = h;
  if (a.nsteps) a.nsteps[b] = (int)N;
}

// the N steps for KN nonzero nodes; one thread per system.  The factor loads
// of the next k are issued before the current k is computed (read-only path,
// no aliasing), so each thread keeps two iterations of loads in flight.
template <int KN>
__global__ void __launch_bounds__(kStepThreads) trid_steps(TArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.batch) return;
  const int N = a.ns[b];
  if (N <= 0) return;
  const int n = a.n;
  const size_t S = a.batch;
  const double h = a.h[b];
  const size_t plane = (size_t)n * S;  // one node's factor array
  const double* __restrict__ lam = a.lam;
  const double* __restrict__ ib = a.ib;
  const double* __restrict__ gg = a.g;
  const double* __restrict__ dl = a.dl;
  const double* __restrict__ dd = a.dd;
  const double* __restrict__ du = a.du;
  double* __restrict__ zs = a.z;
  double cw[KN];
#pragma unroll
  for (int j = 0; j < KN; ++j) cw[j] = a.w[j];
  double z[KN], ln[KN], zn[KN], in[KN], gn[KN];
  for (int q = 0; q < N; ++q) {
    const double* __restrict__ src = q == 0 ? a.V : (((N - q) & 1) == 0 ? a.W : a.sv);
    double* __restrict__ dst = (((N - 1 - q) & 1) == 0) ? a.W : a.sv;
    // forward sweep; windows v_{k-1..k+2}, (B v)_{k-1..k+1}, rows k and k+1 of h A
    double vm = 0.0, v0 = src[b], v1 = n > 1 ? src[S + b] : 0.0, v2 = n > 2 ? src[2 * S + b] : 0.0;
    double hl0 = 0.0, hd0 = 0.0, hu0 = 0.0, hl1 = 0.0, hd1 = 0.0, hu1 = 0.0;
    double bm = 0.0, b0 = 0.0;
    if (a.need_bv) {
      hd0 = h * __ldg(dd + b);
      hu0 = n > 1 ? h * __ldg(du + b) : 0.0;
      if (n > 1) {
        hl1 = h * __ldg(dl + S + b);
        hd1 = h * __ldg(dd + S + b);
        hu1 = n > 2 ? h * __ldg(du + S + b) : 0.0;
      }
      b0 = fma(hd0, v0, hu0 * v1);
    }
#pragma unroll
    for (int j = 0; j < KN; ++j) ln[j] = 0.0;
    for (int k = 0; k < n; ++k) {
      double lc[KN];  // lam of row k (k >= 1), loaded during row k - 1
#pragma unroll
      for (int j = 0; j < KN; ++j) lc[j] = ln[j];
      if (k + 1 < n) {
#pragma unroll
        for (int j = 0; j < KN; ++j) ln[j] = __ldg(lam + j * plane + (size_t)(k + 1) * S + b);
      }
      double b1 = 0.0;
      if (a.need_b2 && k + 1 < n) b1 = fma(hl1, v0, fma(hd1, v1, hu1 * v2));
      double base = a.a0p * v0;
      if (a.need_bv) base = fma(a.d1, b0, base);
      if (a.need_b2) base = fma(a.d2, fma(hl0, bm, fma(hd0, b0, hu0 * b1)), base);
      const double rhs = a.roundoff ? b0 : v0;
      const size_t at = (size_t)k * S + b;
#pragma unroll
      for (int j = 0; j < KN; ++j) {
        z[j] = k == 0 ? rhs : fma(-lc[j], z[j], rhs);
        zs[j * plane + at] = z[j];
      }
      dst[at] = base;
      if (k + 1 < n) {
        vm = v0;
        v0 = v1;
        v1 = v2;
        v2 = k + 3 < n ? src[(size_t)(k + 3) * S + b] : 0.0;
        if (a.need_bv) {
          bm = b0;
          hl0 = hl1;
          hd0 = hd1;
          hu0 = hu1;
          if (k + 2 < n) {
            hl1 = h * __ldg(dl + (size_t)(k + 2) * S + b);
            hd1 = h * __ldg(dd + (size_t)(k + 2) * S + b);
            hu1 = k + 3 < n ? h * __ldg(du + (size_t)(k + 2) * S + b) : 0.0;
          } else {
            hl1 = hd1 = hu1 = 0.0;
          }
          b0 = a.need_b2 ? b1 : fma(hl0, vm, fma(hd0, v0, hu0 * v1));
        }
      }
    }
    // backward sweep and the combination; row k - 1 loaded ahead
    {
      const size_t at = (size_t)(n - 1) * S + b;
#pragma unroll
      for (int j = 0; j < KN; ++j) {
        zn[j] = zs[j * plane + at];
        in[j] = __ldg(ib + j * plane + at);
        gn[j] = 0.0;
      }
    }
    for (int k = n - 1; k >= 0; --k) {
      const size_t at = (size_t)k * S + b;
      double zc[KN], ic[KN], gc[KN];
#pragma unroll
      for (int j = 0; j < KN; ++j) {
        zc[j] = zn[j];
        ic[j] = in[j];
        gc[j] = gn[j];
      }
      if (k > 0) {
        const size_t an = at - S;
#pragma unroll
        for (int j = 0; j < KN; ++j) {
          zn[j] = zs[j * plane + an];
          in[j] = __ldg(ib + j * plane + an);
          gn[j] = __ldg(gg + j * plane + an);
        }
      }
      double acc = dst[at];
#pragma unroll
      for (int j = 0; j < KN; ++j) {
        const double zk = zc[j] * ic[j];
        z[j] = k == n - 1 ? zk : fma(-gc[j], z[j], zk);
        acc = fma(cw[j], z[j], acc);
      }
      dst[at] = acc;
    }
  }
}

template <int KN>
cudaError_t launch_steps(const TArgs& a, cudaStream_t st) {
  const int blocks = (a.batch + kStepThreads - 1) / kStepThreads;
  trid_steps<KN><<<blocks, kStepThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t steps(const TArgs& a, cudaStream_t st) {
  switch (a.kn) {
    case 1: return launch_steps<1>(a, st);
    case 2: return launch_steps<2>(a, st);
    case 3: return launch_steps<3>(a, st);
    case 4: return launch_steps<4>(a, st);
    case 5: return launch_steps<5>(a, st);
    case 6: return launch_steps<6>(a, st);
    case 7: return launch_steps<7>(a, st);
    case 8: return launch_steps<8>(a, st);
    case 9: return launch_steps<9>(a, st);
    case 10: return launch_steps<10>(a, st);
    case 11: return launch_steps<11>(a, st);
    case 12: return launch_steps<12>(a, st);
    case 13: return launch_steps<13>(a, st);
    case 14: return launch_steps<14>(a, st);
    case 15: return launch_steps<15>(a, st);
    default: return launch_steps<16>(a, st);
  }
}

}  // namespace

size_t trid_ws_bytes(int batch, int d, int k) {
  if (batch < 1 || d < 1 || k < 1) return 0;
  return tlay(batch, d, k).total;
}

int trid_run(const TridJob& j, char* msg, size_t len) {
  const TLay L = tlay(j.batch, j.d, j.cf.k);
  if (j.ws_bytes < L.total) {
    snprintf(msg, len, "tridiagonal path: workspace too small");
    return FM_ENOMEM;
  }
  TArgs a = {};
  a.batch = j.batch;
  a.n = j.d;
  a.roundoff = j.form == 0;
  a.dl = j.dl;
  a.dd = j.dd;
  a.du = j.du;
  a.t = j.t;
  a.V = j.V;
  a.W = j.W;
  a.info = j.info;
  a.nsteps = j.nsteps;
  a.anorm = j.anorm;
  a.nsteps_fixed = j.nsteps_fixed;
  a.theta = j.cf.theta;
  a.d1 = j.cf.d1[0];
  a.d2 = j.cf.d2[0];
  // nonzero nodes; the plain form's b_i / (1 - c_i x) = b_i + b_i c_i x / (1 - c_i x)
  // moves b_i of every nonzero node out of the base (a zero node's b_i stays)
  double a0p = j.cf.a0[0];
  int kn = 0;
  for (int i = 0; i < j.cf.k; ++i) {
    const double c = j.cf.c_re[i];
    if (c == 0.0) continue;
    if (j.form == 1) a0p -= j.cf.b_re[0][i];
    a.c[kn] = c;
    a.w[kn] = j.form == 1 ? j.cf.b_re[0][i] : j.cf.b_re[0][i] * c;
    a.idx[kn] = i;
    ++kn;
  }
  a.kn = kn;
  a.a0p = a0p;
  a.need_b2 = a.d2 != 0.0;
  a.need_bv = a.roundoff || a.d1 != 0.0 || a.need_b2;
  char* base = (char*)j.ws;
  a.ns = (int*)(base + L.ns);
  a.h = (double*)(base + L.h);
  a.lam = (double*)(base + L.lam);
  a.ib = (double*)(base + L.ib);
  a.g = (double*)(base + L.g);
  a.z = (double*)(base + L.z);
  a.sv = (double*)(base + L.sv);
  const int blocks = (j.batch + kThreads - 1) / kThreads;
  trid_prep<<<blocks, kThreads, 0, j.st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = steps(a, j.st);
  if (e != cudaSuccess) {
    snprintf(msg, len, "tridiagonal path: %s", cudaGetErrorString(e));
    return FM_ECUDA;
  }
  return FM_OK;
}

}  // namespace fmk
