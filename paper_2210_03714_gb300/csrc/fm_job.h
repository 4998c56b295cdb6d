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
  int conj_pair;  // 1: term i stands for 2 Re(b_i c_i x / (1 - c_i x)) (real
                  //    matrices; complex ones get the set expanded to c, conj(c))
  int pad;
  double c_re[kMaxTerms], c_im[kMaxTerms];
  double b_re[2][kMaxTerms], b_im[2][kMaxTerms];
  double a0[2], d1[2], d2[2];
  double theta;   // min over the functions
};

// One shifted system of a call, in ascending order of its first term.
//  single (quad == 0): M = I - c B; roundoff form Y = M^-1 (c B R), plain form
//    Y = M^-1 R; F_f += w_f Y.
//  quadratic (quad == 1): M = I - u1 B - u2 B^2 after one product B^2, and
//    F_f += M^-1 (g_f I + a_f B + b_f B^2) R.  Two cases:
//    a pair of nodes +c, -c of the roundoff form (u1 = 0, u2 = c^2):
//      b+ cx/(1 - cx) + b- (-cx)/(1 + cx) = ((b+ - b-) c x + (b+ + b-) c^2 x^2)/(1 - c^2 x^2);
//    a term of a conjugate-pair set (u1 = 2 Re c, u2 = -|c|^2, Sec. 1: "one
//    product, x^2, and one inverse" per pair of complex-conjugate roots):
//      2 Re(b cx/(1 - cx)) = (2 Re(bc) x - 2 Re(b) |c|^2 x^2) / (1 - 2 Re(c) x + |c|^2 x^2)
//      2 Re(b/(1 - cx))    = (2 Re(b) - 2 Re(b conj(c)) x) / (same)        (plain form)
struct Sys {
  int node;    // first term index (reported in info for a zero pivot)
  int quad;
  double cr, ci;                    // single: the node
  double u1r, u1i, u2r, u2i;        // quadratic: M = I - u1 B - u2 B^2
  double wr[2], wi[2];              // single: weight per function
  double gr[2], gi[2], ar[2], ai[2], br[2], bi[2];  // quadratic: right-hand side
  // quadratic, the same term through Y = M^-1 - I (the grid paths): with
  // (I + Y) M = I,  (I + Y)(g I + a B + b B^2) = g I + y Y + x (I + Y) B,
  // y = g + b / u2, x = a - b u1 / u2
  double yr[2], yi[2], xr[2], xi[2];
};

// The systems of a set.  fuse_pm: fuse +-c pairs (roundoff form only);
// conjugate-pair terms are always quadratic (their systems stay real).
// base[f]: the multiple of R the combination starts from (a0 in the roundoff
// form; in the plain form a0 minus every weight a nonzero node carries, so the
// singles' b_f M^-1 R and the quadratics' g_f terms add the rest).
FM_HD int plan_systems(const FmCoef& cf, int form, bool fuse_pm, Sys* out, double* base) {
  int ns = 0;
  signed char partner[kMaxTerms];
  for (int i = 0; i < cf.k; ++i) partner[i] = -1;
  for (int f = 0; f < 2; ++f) base[f] = cf.a0[f];
  if (fuse_pm && form == 0 && !cf.conj_pair)
    for (int i = 0; i < cf.k; ++i) {
      if (partner[i] >= 0 || (cf.c_re[i] == 0.0 && cf.c_im[i] == 0.0)) continue;
      for (int q = i + 1; q < cf.k; ++q)
        if (partner[q] < 0 && cf.c_re[q] == -cf.c_re[i] && cf.c_im[q] == -cf.c_im[i]) {
          partner[i] = (signed char)q;
          partner[q] = (signed char)i;
          break;
        }
    }
  for (int i = 0; i < cf.k; ++i) {
    const double cr = cf.c_re[i], ci = cf.c_im[i];
    if (cr == 0.0 && ci == 0.0) continue;  // roundoff: no term; plain: b_i stays in base
    if (partner[i] >= 0 && partner[i] < i) continue;
    Sys& S = out[ns++];
    S.node = i;
    S.quad = 0;
    S.cr = cr;
    S.ci = ci;
    S.u1r = S.u1i = S.u2r = S.u2i = 0.0;
    for (int f = 0; f < 2; ++f) {
      S.wr[f] = cf.b_re[f][i];
      S.wi[f] = cf.b_im[f][i];
      S.gr[f] = S.gi[f] = S.ar[f] = S.ai[f] = S.br[f] = S.bi[f] = 0.0;
      S.yr[f] = S.yi[f] = S.xr[f] = S.xi[f] = 0.0;
    }
    if (cf.conj_pair) {
      for (int f = 0; f < 2; ++f) {
        if (form == 1) base[f] -= 2.0 * cf.b_re[f][i];
      }
      if (ci == 0.0) {  // a real node: 2 Re(b_i) / (1 - c x)
        for (int f = 0; f < 2; ++f) {
          S.wr[f] = 2.0 * cf.b_re[f][i];
          S.wi[f] = 0.0;
        }
        continue;
      }
      S.quad = 1;
      S.u1r = 2.0 * cr;
      S.u2r = -(cr * cr + ci * ci);
      for (int f = 0; f < 2; ++f) {
        const double br = cf.b_re[f][i], bi = cf.b_im[f][i];
        if (form == 0) {
          S.ar[f] = 2.0 * (br * cr - bi * ci);   // 2 Re(b c)
          S.br[f] = 2.0 * br * S.u2r;             // -2 Re(b) |c|^2
        } else {
          S.gr[f] = 2.0 * br;                     // 2 Re(b)
          S.ar[f] = -2.0 * (br * cr + bi * ci);   // -2 Re(b conj(c))
        }
        S.yr[f] = 2.0 * br;                       // both forms
        S.xr[f] = -2.0 * (br * cr + bi * ci);
      }
      continue;
    }
    if (form == 1)
      for (int f = 0; f < 2; ++f) base[f] -= cf.b_re[f][i];
    const int q = partner[i];
    if (q < 0) continue;
    // (b+ - b-) c and (b+ + b-) c^2, complex nodes and weights allowed
    S.quad = 1;
    S.u2r = cr * cr - ci * ci;
    S.u2i = 2.0 * cr * ci;
    for (int f = 0; f < 2; ++f) {
      const double dr = cf.b_re[f][i] - cf.b_re[f][q], di = cf.b_im[f][i] - cf.b_im[f][q];
      const double sr = cf.b_re[f][i] + cf.b_re[f][q], si = cf.b_im[f][i] + cf.b_im[f][q];
      S.ar[f] = dr * cr - di * ci;
      S.ai[f] = dr * ci + di * cr;
      S.br[f] = sr * S.u2r - si * S.u2i;
      S.bi[f] = sr * S.u2i + si * S.u2r;
      S.yr[f] = sr;
      S.yi[f] = si;
      S.xr[f] = S.ar[f];
      S.xi[f] = S.ai[f];
    }
  }
  return ns;
}

enum { JOB_EXPM = 0, JOB_PHI1 = 1, JOB_EXPMV = 2, JOB_PHI1MV = 3, JOB_ADJ = 4, JOB_TRIG = 5 };

// jobs with two functions from one set of resolvents share one scratch layout
FM_HD int layout_kind(int kind) {
  return (kind == JOB_PHI1MV || kind == JOB_TRIG) ? JOB_PHI1 : kind;
}

// opts.s_fixed value of fm_rfun: s = 0 (no range reduction), and info = -5
// when ||tA||_1 exceeds theta (the result is still computed)
constexpr int kSRfun = -2;

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
  size_t Wst, Yst, LamY, UB;                       // adjoint part
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
      // the reverse sweep's c_i lambda_iq (n x kN) and ubar_q (n x N), for the
      // two products that form Bbar after the sweep
      L.LamY = take((size_t)n * k * nmax * elt);
      L.UB = take((size_t)n * nmax * elt);
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
