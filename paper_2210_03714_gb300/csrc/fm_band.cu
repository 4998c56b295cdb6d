// fm_band.cu -- exp(t_b A_b) v_b for a batch of pentadiagonal A_b (half
// bandwidth 2).  Sec. 1 (the dense and sparse cases: a pentadiagonal
// (I + alpha A) x = v is solved in 15d flops, and A v costs 9d) and Sec. 5.1
// (tridiagonal and banded actions): every shifted matrix M_i = I - c_i B of a
// pentadiagonal B is pentadiagonal, so it is factored once per call by banded
// LU without pivoting and solved in every one of the N steps of the action
// recurrence of Sec. 1 (v <- r(B) v, B = (t/N) A).
//
// Same design as the tridiagonal path (fm_trid.cu): one thread per system,
// the batch interleaved (element k of system b at k * batch + b).
//   band_prep   finiteness; eta = ||t A||_1 (column sums, rows in ascending
//               order, as the dense path forms them); N = max(1, ceil(eta /
//               theta)); h = t / N; the factors of every M_i: with m_o the
//               diagonal of M at offset o,
//                 l2_k = m_-2 / beta_{k-2},  l1_k = (m_-1 - l2_k u1_{k-2}) / beta_{k-1},
//                 beta_k = m_0 - l2_k u2_{k-2} - l1_k u1_{k-1},
//                 u1_k = m_+1 - l1_k u2_{k-1},   u2_k = m_+2;
//               stored: l1, l2, 1/beta, g1 = u1/beta, g2 = u2/beta (one
//               division per node and row).  No pivoting: |c_i| ||B||_1 is far
//               below 1/2 at ||B||_1 <= theta, so M_i is diagonally dominant;
//               an exactly zero pivot stops the system with info = i d + row.
//   band_steps  the N steps: forward z_k = rhs_k - l1_k z_{k-1} - l2_k z_{k-2}
//               for all nodes at once (rhs = B v in the roundoff form, v in the
//               plain form), the base a0' v + d1 B v + d2 B^2 v written to the
//               step's output; backward y_k = z_k / beta_k - g1_k y_{k+1} -
//               g2_k y_{k+2} and w_k = base_k + sum_i w_i y_i,k.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/fm.h"
#include "fm_band.h"

namespace fmk {
namespace {

constexpr int kThreads = 128;
constexpr int kStepThreads = 32;

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

// scratch: N and h per system, then l1, l2, 1/beta, g1, g2 and z
// ([node][k][b]), and the second step vector
struct BLay {
  size_t ns, h, l1, l2, ib, g1, g2, z, sv, total;
};
BLay blay(int batch, int d, int k) {
  BLay L;
  size_t o = 0;
  const size_t per = (size_t)k * d * batch * 8;
  L.ns = o; o += up((size_t)batch * 4);
  L.h = o; o += up((size_t)batch * 8);
  L.l1 = o; o += up(per);
  L.l2 = o; o += up(per);
  L.ib = o; o += up(per);
  L.g1 = o; o += up(per);
  L.g2 = o; o += up(per);
  L.z = o; o += up(per);
  L.sv = o; o += up((size_t)d * batch * 8);
  L.total = o;
  return L;
}

struct BArgs {
  int batch, n, kn, roundoff, need_bv, need_b2;
  const double* dg;  // 5 diagonals, offset o = j - 2 at dg + j * n * batch
  const double *t, *V;
  double* W;
  int* info;
  int* nsteps;
  double anorm;
  long long nsteps_fixed;
  double theta, a0p, d1, d2;
  double c[kMaxTerms], w[kMaxTerms];
  int idx[kMaxTerms];
  int* ns;
  double* h;
  double *l1, *l2, *ib, *g1, *g2, *z, *sv;
};

// entry A[k][k + o] of system b (0 outside the matrix)
__device__ __forceinline__ double aent(const BArgs& a, int k, int o, int b) {
  const int c = k + o;
  if (c < 0 || c >= a.n) return 0.0;
  return __ldg(a.dg + ((size_t)(o + 2) * a.n + k) * a.batch + b);
}

__global__ void band_prep(BArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.batch) return;
  const int n = a.n;
  const size_t S = a.batch;
  const double t = a.t[b];
  bool bad = !isfinite(t);
  double eta = 0.0;
  for (int k = 0; k < n; ++k) {
    // column k of t A: rows k-2 .. k+2 in ascending order, A[r][k] = offset k - r of row r
    double s = 0.0;
    for (int r = k - 2; r <= k + 2; ++r) {
      if (r < 0 || r >= n) continue;
      const double v = aent(a, r, k - r, b);
      bad |= !isfinite(v);
      s = __dadd_rn(s, fabs(__dmul_rn(t, v)));
    }
    bad |= !isfinite(a.V[(size_t)k * S + b]);
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
  const size_t plane = (size_t)n * S;
  int zrow[kMaxTerms];
  for (int j = 0; j < a.kn; ++j) zrow[j] = 0;
  for (int j = 0; j < a.kn; ++j) {
    const double c = a.c[j];
    // rows k-1 and k-2: 1/beta, u1, u2
    double ib1 = 0.0, ib2 = 0.0, u1_1 = 0.0, u1_2 = 0.0, u2_1 = 0.0, u2_2 = 0.0;
    for (int k = 0; k < n; ++k) {
      const double mm2 = -__dmul_rn(c, __dmul_rn(h, aent(a, k, -2, b)));
      const double mm1 = -__dmul_rn(c, __dmul_rn(h, aent(a, k, -1, b)));
      const double m0 = __dsub_rn(1.0, __dmul_rn(c, __dmul_rn(h, aent(a, k, 0, b))));
      const double mp1 = -__dmul_rn(c, __dmul_rn(h, aent(a, k, 1, b)));
      const double mp2 = -__dmul_rn(c, __dmul_rn(h, aent(a, k, 2, b)));
      const double l2 = k >= 2 ? __dmul_rn(mm2, ib2) : 0.0;
      const double l1 = k >= 1 ? __dmul_rn(__dsub_rn(mm1, __dmul_rn(l2, u1_2)), ib1) : 0.0;
      const double bet = __dsub_rn(__dsub_rn(m0, __dmul_rn(l2, u2_2)), __dmul_rn(l1, u1_1));
      const double u1 = __dsub_rn(mp1, __dmul_rn(l1, u2_1));
      const double u2 = mp2;
      if (bet == 0.0 && zrow[j] == 0) zrow[j] = k + 1;
      const double r = 1.0 / bet;  // the one division per node and row
      const size_t at = (size_t)j * plane + (size_t)k * S + b;
      a.l1[at] = l1;
      a.l2[at] = l2;
      a.ib[at] = r;
      a.g1[at] = __dmul_rn(u1, r);
      a.g2[at] = __dmul_rn(u2, r);
      ib2 = ib1;
      ib1 = r;
      u1_2 = u1_1;
      u1_1 = u1;
      u2_2 = u2_1;
      u2_1 = u2;
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

// row r of h A as its five diagonals (zero outside the matrix)
__device__ __forceinline__ void load_row(const BArgs& a, int r, int b, double h, double* c) {
#pragma unroll
  for (int o = -2; o <= 2; ++o) c[o + 2] = (r < a.n) ? __dmul_rn(h, aent(a, r, o, b)) : 0.0;
}

// The N steps for KN nonzero nodes; one thread per system.  Sliding windows
// keep v_{k-2..k+4}, the rows k..k+2 of h A and (B v)_{k-2..k+2} in registers
// (B v of row k + 2 is formed at row k, so B^2 v of row k has its five
// neighbours), and every factor is loaded one row ahead on the read-only path.
template <int KN>
__global__ void __launch_bounds__(kStepThreads) band_steps(BArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.batch) return;
  const int N = a.ns[b];
  if (N <= 0) return;
  const int n = a.n;
  const size_t S = a.batch;
  const double h = a.h[b];
  const size_t plane = (size_t)n * S;
  const double* __restrict__ L1 = a.l1;
  const double* __restrict__ L2 = a.l2;
  const double* __restrict__ IB = a.ib;
  const double* __restrict__ G1 = a.g1;
  const double* __restrict__ G2 = a.g2;
  double* __restrict__ zs = a.z;
  double cw[KN];
#pragma unroll
  for (int j = 0; j < KN; ++j) cw[j] = a.w[j];
  for (int q = 0; q < N; ++q) {
    const double* __restrict__ src = q == 0 ? a.V : (((N - q) & 1) == 0 ? a.W : a.sv);
    double* __restrict__ dst = (((N - 1 - q) & 1) == 0) ? a.W : a.sv;
    // windows: vw[i] = v_{k-2+i} (i = 0..6), c0/c1/c2 = rows k, k+1, k+2 of h A,
    // bw[i] = (B v)_{k-2+i} (i = 0..4)
    double vw[7], c0[5], c1[5], c2[5], bw[5];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      const int r = i - 2;
      vw[i] = (r >= 0 && r < n) ? src[(size_t)r * S + b] : 0.0;
    }
    bw[0] = bw[1] = bw[2] = bw[3] = bw[4] = 0.0;
    if (a.need_bv) {
      load_row(a, 0, b, h, c0);
      load_row(a, 1, b, h, c1);
      load_row(a, 2, b, h, c2);
      // (B v)_0 and (B v)_1
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int o = 0; o < 5; ++o) {
        s0 = fma(c0[o], vw[o], s0);      // v_{0 + o - 2}
        s1 = fma(c1[o], vw[o + 1], s1);  // v_{1 + o - 2}
      }
      bw[2] = s0;
      bw[3] = n > 1 ? s1 : 0.0;
    }
    double z1[KN], z2[KN], l1n[KN], l2n[KN];
#pragma unroll
    for (int j = 0; j < KN; ++j) {
      z1[j] = z2[j] = 0.0;
      l1n[j] = l2n[j] = 0.0;  // row 0 has no multipliers
    }
    for (int k = 0; k < n; ++k) {
      const size_t at = (size_t)k * S + b;
      double l1c[KN], l2c[KN];
#pragma unroll
      for (int j = 0; j < KN; ++j) {
        l1c[j] = l1n[j];
        l2c[j] = l2n[j];
      }
      if (k + 1 < n) {
#pragma unroll
        for (int j = 0; j < KN; ++j) {
          l1n[j] = __ldg(L1 + j * plane + at + S);
          l2n[j] = __ldg(L2 + j * plane + at + S);
        }
      }
      double bk = 0.0, b2k = 0.0;
      if (a.need_bv) {
        // (B v)_{k+2} from row k + 2 and v_{k..k+4}
        double s2 = 0.0;
#pragma unroll
        for (int o = 0; o < 5; ++o) s2 = fma(c2[o], vw[o + 2], s2);
        bw[4] = k + 2 < n ? s2 : 0.0;
        bk = bw[2];
        if (a.need_b2) {
#pragma unroll
          for (int o = 0; o < 5; ++o) b2k = fma(c0[o], bw[o], b2k);
        }
      }
      const double v0 = vw[2];
      double base = a.a0p * v0;
      if (a.need_bv) base = fma(a.d1, bk, base);
      if (a.need_b2) base = fma(a.d2, b2k, base);
      const double rhs = a.roundoff ? bk : v0;
#pragma unroll
      for (int j = 0; j < KN; ++j) {
        const double zk = fma(-l2c[j], z2[j], fma(-l1c[j], z1[j], rhs));
        zs[j * plane + at] = zk;
        z2[j] = z1[j];
        z1[j] = zk;
      }
      dst[at] = base;
      // slide the windows one row
#pragma unroll
      for (int i = 0; i < 6; ++i) vw[i] = vw[i + 1];
      vw[6] = k + 5 < n ? src[(size_t)(k + 5) * S + b] : 0.0;
      if (a.need_bv) {
#pragma unroll
        for (int i = 0; i < 4; ++i) bw[i] = bw[i + 1];
#pragma unroll
        for (int o = 0; o < 5; ++o) {
          c0[o] = c1[o];
          c1[o] = c2[o];
        }
        load_row(a, k + 3, b, h, c2);
      }
    }
    // backward sweep and the combination; row k - 1 loaded ahead
    double y1[KN], y2[KN], zn[KN], in[KN], g1n[KN], g2n[KN];
    {
      const size_t at = (size_t)(n - 1) * S + b;
#pragma unroll
      for (int j = 0; j < KN; ++j) {
        y1[j] = y2[j] = 0.0;
        zn[j] = zs[j * plane + at];
        in[j] = __ldg(IB + j * plane + at);
        g1n[j] = __ldg(G1 + j * plane + at);
        g2n[j] = __ldg(G2 + j * plane + at);
      }
    }
    for (int k = n - 1; k >= 0; --k) {
      const size_t at = (size_t)k * S + b;
      double zc[KN], ic[KN], g1c[KN], g2c[KN];
#pragma unroll
      for (int j = 0; j < KN; ++j) {
        zc[j] = zn[j];
        ic[j] = in[j];
        g1c[j] = g1n[j];
        g2c[j] = g2n[j];
      }
      if (k > 0) {
        const size_t an = at - S;
#pragma unroll
        for (int j = 0; j < KN; ++j) {
          zn[j] = zs[j * plane + an];
          in[j] = __ldg(IB + j * plane + an);
          g1n[j] = __ldg(G1 + j * plane + an);
          g2n[j] = __ldg(G2 + j * plane + an);
        }
      }
      double acc = dst[at];
#pragma unroll
      for (int j = 0; j < KN; ++j) {
        const double yk = fma(-g2c[j], y2[j], fma(-g1c[j], y1[j], zc[j] * ic[j]));
        y2[j] = y1[j];
        y1[j] = yk;
        acc = fma(cw[j], yk, acc);
      }
      dst[at] = acc;
    }
  }
}

template <int KN>
cudaError_t launch_steps(const BArgs& a, cudaStream_t st) {
  const int blocks = (a.batch + kStepThreads - 1) / kStepThreads;
  band_steps<KN><<<blocks, kStepThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t steps(const BArgs& a, cudaStream_t st) {
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

size_t penta_ws_bytes(int batch, int d, int k) {
  if (batch < 1 || d < 1 || k < 1) return 0;
  return blay(batch, d, k).total;
}

int penta_run(const PentaJob& j, char* msg, size_t len) {
  const BLay L = blay(j.batch, j.d, j.cf.k);
  if (j.ws_bytes < L.total) {
    snprintf(msg, len, "pentadiagonal path: workspace too small");
    return FM_ENOMEM;
  }
  BArgs a = {};
  a.batch = j.batch;
  a.n = j.d;
  a.roundoff = j.form == 0;
  a.dg = j.diags;
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
  // nonzero nodes; the plain form moves b_i of every nonzero node out of the base
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
  a.l1 = (double*)(base + L.l1);
  a.l2 = (double*)(base + L.l2);
  a.ib = (double*)(base + L.ib);
  a.g1 = (double*)(base + L.g1);
  a.g2 = (double*)(base + L.g2);
  a.z = (double*)(base + L.z);
  a.sv = (double*)(base + L.sv);
  const int blocks = (j.batch + kThreads - 1) / kThreads;
  band_prep<<<blocks, kThreads, 0, j.st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = steps(a, j.st);
  if (e != cudaSuccess) {
    snprintf(msg, len, "pentadiagonal path: %s", cudaGetErrorString(e));
    return FM_ECUDA;
  }
  return FM_OK;
}

}  // namespace fmk
