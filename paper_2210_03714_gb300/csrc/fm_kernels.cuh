// fm_kernels.cuh -- persistent batched kernels: one CTA owns one matrix at a
// time and runs every step of the method on it (S. Blanes, arXiv:2210.03714):
//
//   a1  eta = ||tA||_1 (or anorm |t|); s = smallest with eta/2^s <= theta
//       (N = ceil(eta/theta) for actions)                      Sec. 1, Sec. 3
//   a2  B = tA/2^s  (B = (t/N) A for actions)                  Sec. 1
//   a3  M_i = I - c_i B, LU with partial pivoting              Sec. 1, Sec. 2
//   a4  Y_i = M_i^{-1} (c_i B R)  (roundoff form)              Eq. ParallRoundOff, Frac10R
//   a5  mixed precision: factor/solve in single, then refine
//       Y_i += M_i^{-1} (c_i B R - M_i Y_i) with the residual in double
//   a6  F = a0 R + d1 B R + d2 B^2 R + sum_i b_i Y_i          Eq. ParallRoundOff, Frac10
//   a7  s squarings F <- F F; phi_1 doubling (Phi, E) <- ((E+I)Phi/2, E^2);
//       or N steps of the action with the factorizations reused   Sec. 1
//
// The element-wise steps are written in the same order as the textbook
// definition (C = c_i B rounded once, M = I - C, F = F + b_i Y) so that the
// only rounding differences against a plain double-precision evaluation come
// from the factorizations and the products.
#pragma once
#include "cta_la.cuh"
#include "fm_job.h"
#include "ozaki.cuh"

namespace fmk {

template <class T>
__device__ __forceinline__ T tdiag(int r, int c) {
  return r == c ? Tr<T>::one() : Tr<T>::zero();
}

// b * y for a real-or-complex weight stored as (re, im)
template <class T> __device__ __forceinline__ T wmul(double br, double bi, T y);
template <> __device__ __forceinline__ double wmul<double>(double br, double, double y) {
  return __dmul_rn(br, y);
}
template <> __device__ __forceinline__ zd wmul<zd>(double br, double bi, zd y) {
  return Tr<zd>::mul(zd{br, bi}, y);
}

__device__ __forceinline__ int select_s(double eta, double theta) {
  int s = 0;
  while (eta > ldexp(theta, s) && s < 1023) ++s;
  return s;
}

__device__ __forceinline__ double tscale(double a, int s) { return ldexp(a, -s); }
__device__ __forceinline__ zd tscale(zd a, int s) { return {ldexp(a.x, -s), ldexp(a.y, -s)}; }

// exact rounding error of fl(1 - c): returns fl(1 - c) - (1 - c)  (TwoSum)
__device__ __forceinline__ double diag_err(double c) {
  double a = 1.0, b = -c;
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double err = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return -err;
}
__device__ __forceinline__ double diag_err(zd c) { return diag_err(c.x); }

template <class T> __device__ __forceinline__ T dscale(double dr, T y);
template <> __device__ __forceinline__ double dscale<double>(double dr, double y) { return __dmul_rn(dr, y); }
template <> __device__ __forceinline__ zd dscale<zd>(double dr, zd y) { return {__dmul_rn(dr, y.x), __dmul_rn(dr, y.y)}; }

template <class T> __device__ __forceinline__ typename Tr<T>::R tmag(T a) { return Tr<T>::mag(a); }

// ---------------------------------------------------------------------------
// P = X Y accurate to double: the Ozaki tensor-core product when the CTA has a
// tensor-core context (real mixed path), else the double-precision CTA GEMM.
// Returns nonzero when a tensor-core wait timed out.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ int prod(oz::Ctx* oc, int M, int N, int K, const T* X, int ldx,
                                    const T* Y, int ldy, T* P, int ldp, char* smem,
                                    bool reuse_x = false) {
  if constexpr (sizeof(T) == 8) {
    if (oc) return oz::gemm(*oc, M, N, K, (const double*)X, ldx, (const double*)Y, ldy,
                            (double*)P, ldp, reuse_x);
  }
  cta_gemm<T>(M, N, K, (typename Tr<T>::R)1, X, ldx, Y, ldy, (typename Tr<T>::R)0, P, ldp,
              (T*)(smem + 256));
  return 0;
}

// point the tensor-core context at this matrix's digit-plane scratch
__device__ __forceinline__ void oz_bind(oz::Ctx* oc, char* ws, const WsLayout& L) {
  if (!oc) return;
  if (threadIdx.x == 0) {
    oc->gx = (unsigned char*)(ws + L.gx);
    oc->gy = (unsigned char*)(ws + L.gy);
    oc->ex = (int*)(ws + L.ex);
    oc->fy = (int*)(ws + L.fy);
  }
  __syncthreads();
}

// LU solve with the right-hand sides staged in shared memory when they fit
template <class T, int NB>
__device__ __forceinline__ void solve_lu(const FmJob& J, int n, const T* LU, const int* piv, int m,
                                         T* X, char* smem) {
  const size_t budget = J.smem_avail / sizeof(T);
  if (budget > 0 && (size_t)16 * n + (size_t)NT * 16 + 64 <= budget)
    cta_getrs_ll<T>(n, LU, n, piv, m, X, m, (T*)smem);
  else
    cta_getrs<T, NB>(n, LU, n, piv, m, X, m, (T*)smem);
}

// ---------------------------------------------------------------------------
// One shifted solve: Y = M^{-1} RHS with M = I - C (+ exact diagonal rounding
// D), factors LU (type TL) already computed.  Double precision: one solve in
// T.  Mixed: solve in TL, then max_ir refinement steps with the residual
// RHS - M Y = ((RHS - Y) + C Y) - D Y evaluated in T.  Returns the last
// relative correction (or -1 when none was made).
// ---------------------------------------------------------------------------
template <class T, class TL, int NB>
__device__ __noinline__ double shifted_solve(const FmJob& J, int n, int m, const T* C, const double* D,
                                const TL* LU, const int* piv, const T* RHS, T* Y, T* P, TL* RL,
                                char* smem, oz::Ctx* oc, int* terr) {
  using TT = Tr<T>;
  using R = typename TT::R;
  const int tid = threadIdx.x;
  const size_t nm = (size_t)n * m;
  if (sizeof(TL) == sizeof(T) && J.precision == 0) {
    for (size_t e = tid; e < nm; e += NT) Y[e] = RHS[e];
    __syncthreads();
    solve_lu<T, NB>(J, n, (const T*)LU, piv, m, Y, smem);
    return -1.0;
  }
  for (size_t e = tid; e < nm; e += NT) RL[e] = cvt<TL, T>(RHS[e]);
  __syncthreads();
  solve_lu<TL, NB>(J, n, LU, piv, m, RL, smem);
  for (size_t e = tid; e < nm; e += NT) Y[e] = cvt<T, TL>(RL[e]);
  __syncthreads();
  double q = -1.0;
  R* red = (R*)(smem + 64);
  for (int it = 0; it < J.max_ir; ++it) {
    // P = C Y  (double-accurate product)
    *terr |= prod<T>(oc, n, m, n, C, n, Y, m, P, m, smem, it > 0);
    for (size_t e = tid; e < nm; e += NT) {
      int r = (int)(e / m);
      T v = TT::add(TT::sub(RHS[e], Y[e]), P[e]);
      v = TT::sub(v, dscale<T>(D[r], Y[e]));
      RL[e] = cvt<TL, T>(v);
    }
    __syncthreads();
    solve_lu<TL, NB>(J, n, LU, piv, m, RL, smem);
    R dmax = 0, ymax = 0;
    for (size_t e = tid; e < nm; e += NT) {
      T dl = cvt<T, TL>(RL[e]);
      T y = TT::add(Y[e], dl);
      Y[e] = y;
      dmax = fmax(dmax, tmag(dl));
      ymax = fmax(ymax, tmag(y));
    }
    __syncthreads();
    dmax = cta_max<R>(dmax, red);
    ymax = cta_max<R>(ymax, red);
    q = ymax > 0 ? (double)(dmax / ymax) : (double)dmax;
  }
  return q;
}

template <class T, class TL>
__device__ __forceinline__ void build_shift(int n, double cre, double cim, const T* B, T* C, TL* LU,
                                            double* D, bool mixed) {
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += NT) {
    int r = e / n, c = e % n;
    T cv = wmul<T>(cre, cim, B[e]);  // C = c_i B, one rounding
    C[e] = cv;
    T mv = Tr<T>::sub(tdiag<T>(r, c), cv);  // M = I - C
    LU[e] = cvt<TL, T>(mv);
    if (r == c) D[r] = mixed ? diag_err(cv) : 0.0;
  }
  __syncthreads();
}

// C = u1 B + u2 B2 (each product rounded once; C = u2 B2 when u1 = 0), M = I - C
template <class T, class TL>
__device__ __forceinline__ void build_shift2(int n, double u1r, double u1i, const T* B, double u2r,
                                             double u2i, const T* B2, T* C, TL* LU, double* D,
                                             bool mixed) {
  const int tid = threadIdx.x;
  const bool one = u1r == 0.0 && u1i == 0.0;
  for (int e = tid; e < n * n; e += NT) {
    int r = e / n, c = e % n;
    T cv = wmul<T>(u2r, u2i, B2[e]);
    if (!one) cv = Tr<T>::add(wmul<T>(u1r, u1i, B[e]), cv);
    C[e] = cv;
    T mv = Tr<T>::sub(tdiag<T>(r, c), cv);
    LU[e] = cvt<TL, T>(mv);
    if (r == c) D[r] = mixed ? diag_err(cv) : 0.0;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// matrix functions: exp (JOB_EXPM), phi_1 with exp (JOB_PHI1, JOB_PHI1MV)
// ---------------------------------------------------------------------------
template <class T, class TL, int NB>
__device__ __noinline__ void run_matfun(const FmJob& J, const FmCoef& cf, int b, char* ws, char* smem,
                                        oz::Ctx* oc, Sys* plan) {
  using TT = Tr<T>;
  using R = typename TT::R;
  const int tid = threadIdx.x;
  const bool batched = J.d != nullptr;
  const int n = batched ? J.d[b] : J.d1;
  const int64_t off = batched ? J.off[b] : 0;
  const int lda = batched ? n : J.lda, ldf = batched ? n : J.ldf, lde = batched ? n : J.lde;
  const double t = J.t ? J.t[b] : J.t1;
  const bool mixed = J.precision != 0;
  const bool two = (J.kind != JOB_EXPM);
  const bool trig = J.kind == JOB_TRIG;  // cos (F) and sin (Ph)
  const WsLayout L = ws_layout(layout_kind(J.kind), n, J.m, cf.k, sizeof(T), sizeof(TL), 0,
                               oc != nullptr);
  oz_bind(oc, ws, L);
  int terr = 0;
  T* B = (T*)(ws + L.B);
  T* C = (T*)(ws + L.C);
  T* Y = (T*)(ws + L.Y);
  T* T1 = (T*)(ws + L.T1);
  T* F = (T*)(ws + L.F);
  T* Ph = (T*)(ws + L.Phi);
  TL* LU = (TL*)(ws + L.LU);
  TL* RL = (TL*)(ws + L.RL);
  int* piv = (int*)(ws + L.piv);
  double* D = (double*)(ws + L.D);
  R* red = (R*)smem;
  int* redi = (int*)(smem + 128);
  const T* A = (const T*)J.A + off;

  // a1/a2: B = tA, finiteness, eta = ||tA||_1, s, B = tA/2^s
  int bad = !isfinite(t);
  for (int e = tid; e < n * n; e += NT) {
    int r = e / n, c = e % n;
    T a = A[(size_t)r * lda + c];
    bad |= !TT::finite(a);
    B[e] = TT::rscale(a, t);
  }
  __syncthreads();
  bad = cta_or(bad, redi);
  R cmax = 0;
  for (int c = tid; c < n; c += NT) {
    R s = 0;
    for (int r = 0; r < n; ++r) s += tmag(B[r * n + c]);
    cmax = (s > cmax || isnan(s)) ? s : cmax;
  }
  cmax = cta_max<R>(cmax, red);
  int info = 0;
  if (bad) info = -2;
  const double eta = J.anorm > 0 ? J.anorm * fabs(t) : (double)cmax;
  const int s = J.s_fixed >= 0 ? J.s_fixed : (J.s_fixed == kSRfun ? 0 : select_s(eta, cf.theta));
  for (int e = tid; e < n * n; e += NT) B[e] = tscale(B[e], s);
  // a3-a6 plan: one system per nonzero node; in the roundoff form a pair of
  // nodes +c, -c shares one system I - c^2 B^2, and a term of a conjugate-pair
  // set is one real system I - 2 Re(c) B + |c|^2 B^2 (Sec. 1: one product, x^2,
  // and one inverse per pair of roots)
  // (the plan lives in shared memory, filled by one thread)
  Sys* sys = plan;
  double* pbase = (double*)(plan + kMaxTerms);
  int* pn = (int*)(pbase + 2);
  if (tid == 0) *pn = plan_systems(cf, J.form, true, sys, pbase);
  __syncthreads();
  const int nsys = *pn;
  const double base[2] = {pbase[0], pbase[1]};
  bool any_quad = false;
  for (int q = 0; q < nsys; ++q) any_quad |= sys[q].quad != 0;
  const bool hyb = cf.d1[0] != 0 || cf.d2[0] != 0 || (two && (cf.d1[1] != 0 || cf.d2[1] != 0));
  T* B2 = (T*)(ws + L.B2);
  const bool need_b2 = cf.d2[0] != 0 || (two && cf.d2[1] != 0) || any_quad;
  if (need_b2) terr |= prod<T>(oc, n, n, n, B, n, B, n, B2, n, smem);
  // a6 (first part): F = base I (+ d1 B + d2 B^2) for each function
  for (int e = tid; e < n * n; e += NT) {
    int r = e / n, c = e % n;
    for (int f = 0; f < (two ? 2 : 1); ++f) {
      T v = TT::rscale(tdiag<T>(r, c), base[f]);
      if (hyb) {
        if (cf.d1[f] != 0) v = TT::add(v, TT::rscale(B[e], cf.d1[f]));
        if (cf.d2[f] != 0) v = TT::add(v, TT::rscale(B2[e], cf.d2[f]));
      }
      (f == 0 ? F : Ph)[e] = v;
    }
  }
  __syncthreads();
  double qmax = -1.0;
  const bool any_shift = nsys > 0;
  // a3-a6: the shifted solves, ascending first term
  for (int q = 0; q < nsys && info == 0; ++q) {
    const Sys& S = sys[q];
    if (S.quad) {
      // one system M = I - u1 B - u2 B^2; per function the right-hand side
      // X = g I + a B + b B^2, and F += M^-1 X
      build_shift2<T, TL>(n, S.u1r, S.u1i, B, S.u2r, S.u2i, B2, C, LU, D, mixed);
      int fi = cta_getrf<TL, NB>(n, LU, n, piv, (TL*)smem);
      if (fi) { info = S.node * n + fi; break; }
      for (int f = 0; f < (two ? 2 : 1); ++f) {
        for (int e = tid; e < n * n; e += NT) {
          T v = wmul<T>(S.ar[f], S.ai[f], B[e]);
          if (S.br[f] != 0.0 || S.bi[f] != 0.0) v = TT::add(v, wmul<T>(S.br[f], S.bi[f], B2[e]));
          if (e / n == e % n && (S.gr[f] != 0.0 || S.gi[f] != 0.0))
            v = TT::add(v, wmul<T>(S.gr[f], S.gi[f], TT::one()));
          T1[e] = v;
        }
        __syncthreads();
        double qq = shifted_solve<T, TL, NB>(J, n, n, C, D, LU, piv, T1, Y, (T*)(ws + L.T2), RL,
                                             smem, oc, &terr);
        qmax = fmax(qmax, qq);
        T* Fx = f == 0 ? F : Ph;
        for (int e = tid; e < n * n; e += NT) Fx[e] = TT::add(Fx[e], Y[e]);
        __syncthreads();
      }
      continue;
    }
    build_shift<T, TL>(n, S.cr, S.ci, B, C, LU, D, mixed);
    int fi = cta_getrf<TL, NB>(n, LU, n, piv, (TL*)smem);
    if (fi) { info = S.node * n + fi; break; }
    // right-hand side: C (roundoff form) or I (plain form), kept in T1
    for (int e = tid; e < n * n; e += NT) {
      int r = e / n, c = e % n;
      T1[e] = J.form == 1 ? tdiag<T>(r, c) : C[e];
    }
    __syncthreads();
    double qq = shifted_solve<T, TL, NB>(J, n, n, C, D, LU, piv, T1, Y, (T*)(ws + L.T2), RL, smem,
                                         oc, &terr);
    qmax = fmax(qmax, qq);
    for (int e = tid; e < n * n; e += NT)
      for (int f = 0; f < (two ? 2 : 1); ++f) {
        T* Fx = f == 0 ? F : Ph;
        Fx[e] = TT::add(Fx[e], wmul<T>(S.wr[f], S.wi[f], Y[e]));
      }
    __syncthreads();
  }
  if (info == 0 && mixed && J.ir_tol > 0 && any_shift && (J.max_ir == 0 || qmax > J.ir_tol)) info = -1;
  // a7: squarings / doublings
  T* T2 = (T*)(ws + L.T2);
  if ((info == 0 || info == -1) && oc != nullptr && s > 0) {
    // Tensor-core products are accurate relative to the largest entry of each
    // row and column, so square the deviation from the identity instead of
    // F itself: (I + E)^2 = I + (2E + E E); for phi_1 with Phi = I + Psi,
    // (E_F + I) Phi / 2 = I + (Psi + E/2 + E Psi / 2).  Same recurrence.
    // cos and sin (double angle, Sec. 1) with C = I + X: 2 C^2 - I = I + (4X + 2 X X)
    // and 2 S C = 2S + 2 X S (S and X commute: both are functions of B).
    for (int r = tid; r < n; r += NT) {
      F[r * n + r] = TT::sub(F[r * n + r], TT::one());
      if (two && !trig) Ph[r * n + r] = TT::sub(Ph[r * n + r], TT::one());
    }
    __syncthreads();
    for (int q = 0; q < s; ++q) {
      if (two) terr |= prod<T>(oc, n, n, n, F, n, Ph, n, T1, n, smem);
      terr |= prod<T>(oc, n, n, n, F, n, F, n, T2, n, smem);
      for (int e = tid; e < n * n; e += NT) {
        const T E = F[e];
        if (trig) {
          Ph[e] = TT::add(TT::rscale(Ph[e], 2.0), TT::rscale(T1[e], 2.0));
          F[e] = TT::add(TT::rscale(E, 4.0), TT::rscale(T2[e], 2.0));
          continue;
        }
        if (two) Ph[e] = TT::add(TT::add(Ph[e], TT::rscale(E, 0.5)), TT::rscale(T1[e], 0.5));
        F[e] = TT::add(TT::rscale(E, 2.0), T2[e]);
      }
      __syncthreads();
    }
    for (int r = tid; r < n; r += NT) {
      F[r * n + r] = TT::add(F[r * n + r], TT::one());
      if (two && !trig) Ph[r * n + r] = TT::add(Ph[r * n + r], TT::one());
    }
  } else if (info == 0 || info == -1) {
    for (int q = 0; q < s; ++q) {
      if (!two) {
        terr |= prod<T>(oc, n, n, n, F, n, F, n, T1, n, smem);
        T* tmp = F; F = T1; T1 = tmp;
      } else if (trig) {
        // (C, S) <- (2 C^2 - I, 2 S C)
        terr |= prod<T>(oc, n, n, n, Ph, n, F, n, T1, n, smem);
        terr |= prod<T>(oc, n, n, n, F, n, F, n, T2, n, smem);
        for (int e = tid; e < n * n; e += NT) {
          Ph[e] = TT::rscale(T1[e], 2.0);
          F[e] = TT::sub(TT::rscale(T2[e], 2.0), tdiag<T>(e / n, e % n));
        }
        __syncthreads();
      } else {
        // Phi <- (E + I) Phi / 2, then E <- E E
        for (int r = tid; r < n; r += NT) F[r * n + r] = TT::add(F[r * n + r], TT::one());
        __syncthreads();
        terr |= prod<T>(oc, n, n, n, F, n, Ph, n, T1, n, smem);
        for (int e = tid; e < n * n; e += NT) Ph[e] = TT::rscale(T1[e], 0.5);
        for (int r = tid; r < n; r += NT) F[r * n + r] = TT::sub(F[r * n + r], TT::one());
        __syncthreads();
        terr |= prod<T>(oc, n, n, n, F, n, F, n, T2, n, smem);
        T* tmp = F; F = T2; T2 = tmp;
      }
    }
  }
  __syncthreads();
  if (J.s_fixed == kSRfun && info == 0 && !(eta <= cf.theta)) info = -5;
  // outputs
  if (J.kind == JOB_TRIG) {
    T* Co = (T*)J.F + off;
    for (int e = tid; e < n * n; e += NT) Co[(size_t)(e / n) * ldf + e % n] = F[e];
    if (J.E) {
      T* So = (T*)J.E + off;
      for (int e = tid; e < n * n; e += NT) So[(size_t)(e / n) * lde + e % n] = Ph[e];
    }
  } else if (J.kind == JOB_EXPM) {
    T* Fo = (T*)J.F + off;
    for (int e = tid; e < n * n; e += NT) Fo[(size_t)(e / n) * ldf + e % n] = F[e];
  } else if (J.kind == JOB_PHI1) {
    T* Po = (T*)J.F + off;
    for (int e = tid; e < n * n; e += NT) Po[(size_t)(e / n) * ldf + e % n] = Ph[e];
    if (J.E) {
      T* Eo = (T*)J.E + off;
      for (int e = tid; e < n * n; e += NT) Eo[(size_t)(e / n) * lde + e % n] = F[e];
    }
  } else {  // PHI1MV: W = Phi V
    const int m = J.m;
    const int64_t vo = batched ? J.voff[b] : 0;
    const int ldv = batched ? m : J.ldv, ldw = batched ? m : J.ldw;
    terr |= prod<T>(oc, n, m, n, Ph, n, (const T*)J.V + vo, ldv, (T*)J.W + vo, ldw, smem);
  }
  if (terr && (info == 0 || info == -1)) info = -7;
  if (tid == 0) {
    if (J.info) J.info[b] = info;
    if (J.sN) J.sN[b] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// action: W = exp(tA) V (JOB_EXPMV)
// ---------------------------------------------------------------------------
template <class T, class TL, int NB>
__device__ __noinline__ void run_action(const FmJob& J, const FmCoef& cf, int b, char* ws, char* smem,
                                        oz::Ctx* oc, Sys* plan) {
  using TT = Tr<T>;
  using R = typename TT::R;
  const int tid = threadIdx.x;
  const bool batched = J.d != nullptr;
  const int n = batched ? J.d[b] : J.d1;
  const int m = J.m;
  const int64_t off = batched ? J.off[b] : 0;
  const int64_t vo = batched ? J.voff[b] : 0;
  const int lda = batched ? n : J.lda;
  const int ldv = batched ? m : J.ldv, ldw = batched ? m : J.ldw;
  const double t = J.t ? J.t[b] : J.t1;
  const bool mixed = J.precision != 0;
  const int k = cf.k;
  const WsLayout L = ws_layout(JOB_EXPMV, n, m, k, sizeof(T), sizeof(TL), 0, oc != nullptr);
  oz_bind(oc, ws, L);
  int terr = 0;
  T* B = (T*)(ws + L.B);
  T* Y = (T*)(ws + L.Y);
  T* P = (T*)(ws + L.T1);
  TL* RL = (TL*)(ws + L.RL);
  T* Wc = (T*)(ws + L.Wc);
  T* Wn = (T*)(ws + L.Wn);
  T* U = (T*)(ws + L.U);
  T* U2 = (T*)(ws + L.U2);
  T* RHS = (T*)(ws + L.RHS);
  R* red = (R*)smem;
  int* redi = (int*)(smem + 128);
  const T* A = (const T*)J.A + off;
  const T* V = (const T*)J.V + vo;
  const size_t nm = (size_t)n * m;

  int bad = !isfinite(t);
  for (int e = tid; e < n * n; e += NT) {
    int r = e / n, c = e % n;
    T a = A[(size_t)r * lda + c];
    bad |= !TT::finite(a);
    B[e] = TT::rscale(a, t);
  }
  for (size_t e = tid; e < nm; e += NT) {
    T v = V[(e / m) * ldv + e % m];
    bad |= !TT::finite(v);
    Wc[e] = v;
  }
  __syncthreads();
  bad = cta_or(bad, redi);
  R cmax = 0;
  for (int c = tid; c < n; c += NT) {
    R s = 0;
    for (int r = 0; r < n; ++r) s += tmag(B[r * n + c]);
    cmax = (s > cmax || isnan(s)) ? s : cmax;
  }
  cmax = cta_max<R>(cmax, red);
  int info = bad ? -2 : 0;
  const double eta = J.anorm > 0 ? J.anorm * fabs(t) : (double)cmax;
  long long N = J.nsteps;
  if (N <= 0) {
    double qn = ceil(eta / cf.theta);
    N = qn < 1.0 ? 1 : (long long)qn;
  }
  const double h = t / (double)N;
  for (int e = tid; e < n * n; e += NT) {
    int r = e / n, c = e % n;
    B[e] = TT::rscale(A[(size_t)r * lda + c], h);
  }
  __syncthreads();
  // one system per nonzero node (the +-c pairs stay apart here: each step's
  // solves already share the one product B W); a term of a conjugate-pair set
  // is one real system I - 2 Re(c) B + |c|^2 B^2 (Sec. 1)
  Sys* sys = plan;
  double* pbase = (double*)(plan + kMaxTerms);
  int* pn = (int*)(pbase + 2);
  if (tid == 0) *pn = plan_systems(cf, J.form, false, sys, pbase);
  __syncthreads();
  const int nsys = *pn;
  const double base = pbase[0];
  bool any_quad = false, quad_b2 = false;
  for (int q = 0; q < nsys; ++q) {
    any_quad |= sys[q].quad != 0;
    quad_b2 |= sys[q].quad != 0 && (sys[q].br[0] != 0.0 || sys[q].bi[0] != 0.0);
  }
  T* B2 = (T*)(ws + L.C);  // B^2 for the quadratic systems (C is unused here)
  if (any_quad && info == 0) terr |= prod<T>(oc, n, n, n, B, n, B, n, B2, n, smem);
  // a3: factor every shifted matrix once (slot = the system's first term)
  for (int q = 0; q < nsys && info == 0; ++q) {
    const Sys& S = sys[q];
    const int i = S.node;
    T* Ci = (T*)(ws + L.Cs) + (size_t)i * n * n;
    TL* LUi = (TL*)(ws + L.LUs) + (size_t)i * n * n;
    int* pivi = (int*)(ws + L.pivs) + (size_t)i * n;
    double* Di = (double*)(ws + L.Ds) + (size_t)i * n;
    if (S.quad) build_shift2<T, TL>(n, S.u1r, S.u1i, B, S.u2r, S.u2i, B2, Ci, LUi, Di, mixed);
    else build_shift<T, TL>(n, S.cr, S.ci, B, Ci, LUi, Di, mixed);
    int fi = cta_getrf<TL, NB>(n, LUi, n, pivi, (TL*)smem);
    if (fi) info = i * n + fi;
  }
  double qmax = -1.0;
  const bool any_shift = nsys > 0;
  const bool need_u2 = cf.d2[0] != 0 || quad_b2;
  // a4-a7: N steps W <- r(B) W
  for (long long q = 0; q < N && info == 0; ++q) {
    terr |= prod<T>(oc, n, m, n, B, n, Wc, m, U, m, smem);
    if (need_u2) terr |= prod<T>(oc, n, m, n, B, n, U, m, U2, m, smem);
    for (size_t e = tid; e < nm; e += NT) {
      T v = TT::rscale(Wc[e], base);
      if (cf.d1[0] != 0) v = TT::add(v, TT::rscale(U[e], cf.d1[0]));
      if (cf.d2[0] != 0) v = TT::add(v, TT::rscale(U2[e], cf.d2[0]));
      Wn[e] = v;
    }
    __syncthreads();
    for (int qs = 0; qs < nsys; ++qs) {
      const Sys& S = sys[qs];
      const int i = S.node;
      const T* Ci = (const T*)(ws + L.Cs) + (size_t)i * n * n;
      const TL* LUi = (const TL*)(ws + L.LUs) + (size_t)i * n * n;
      const int* pivi = (const int*)(ws + L.pivs) + (size_t)i * n;
      const double* Di = (const double*)(ws + L.Ds) + (size_t)i * n;
      if (S.quad) {
        // right-hand side g W + a B W + b B^2 W
        for (size_t e = tid; e < nm; e += NT) {
          T v = wmul<T>(S.ar[0], S.ai[0], U[e]);
          if (S.br[0] != 0.0 || S.bi[0] != 0.0) v = TT::add(v, wmul<T>(S.br[0], S.bi[0], U2[e]));
          if (S.gr[0] != 0.0 || S.gi[0] != 0.0) v = TT::add(v, wmul<T>(S.gr[0], S.gi[0], Wc[e]));
          RHS[e] = v;
        }
      } else {
        for (size_t e = tid; e < nm; e += NT) RHS[e] = J.form == 1 ? Wc[e] : wmul<T>(S.cr, S.ci, U[e]);
      }
      __syncthreads();
      double qq = shifted_solve<T, TL, NB>(J, n, m, Ci, Di, LUi, pivi, RHS, Y, P, RL, smem, oc,
                                           &terr);
      qmax = fmax(qmax, qq);
      if (S.quad)
        for (size_t e = tid; e < nm; e += NT) Wn[e] = TT::add(Wn[e], Y[e]);
      else
        for (size_t e = tid; e < nm; e += NT) Wn[e] = TT::add(Wn[e], wmul<T>(S.wr[0], S.wi[0], Y[e]));
      __syncthreads();
    }
    T* tmp = Wc; Wc = Wn; Wn = tmp;
  }
  if (info == 0 && mixed && J.ir_tol > 0 && any_shift && (J.max_ir == 0 || qmax > J.ir_tol)) info = -1;
  if (terr && (info == 0 || info == -1)) info = -7;
  T* Wo = (T*)J.W + vo;
  for (size_t e = tid; e < nm; e += NT) Wo[(e / m) * ldw + e % m] = Wc[e];
  if (tid == 0) {
    if (J.info) J.info[b] = info;
    if (J.sN) J.sN[b] = (int)(N > 0x7fffffff ? 0x7fffffff : N);
  }
  __syncthreads();
}

// y = s M x, M n x n row-major (one warp per row); y must not alias x
__device__ __forceinline__ void cta_gemv(int n, const double* M, const double* x, double s,
                                         double* y) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = w; r < n; r += NT / 32) {
    double acc = 0.0;
    for (int c = lane; c < n; c += 32) acc = fma(M[(size_t)r * n + c], x[c], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[r] = s * acc;
  }
  __syncthreads();
}

// k stacked products y_i = s_i M_i x (M_i n x n row-major, M_i at M + i n n,
// y_i at y + i n), one warp per row of the k n stacked rows; a block with
// s_i = 0 gives y_i = 0 without reading M_i.  y must not alias x.
__device__ __forceinline__ void cta_gemv_stack(int n, int k, const double* M, const double* x,
                                               const double* s, double* y) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = w; r < k * n; r += NT / 32) {
    const double si = s[r / n];
    double acc = 0.0;
    if (si != 0.0)
      for (int c = lane; c < n; c += 32) acc = fma(M[(size_t)r * n + c], x[c], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[r] = si * acc;
  }
  __syncthreads();
}

// k stacked transposed products y_i = s_i M_i^T x, one output (i, c) per
// thread and pass, four outputs per thread in one sweep over the rows (four
// independent sums); a block with s_i = 0 gives y_i = 0.
__device__ __forceinline__ void cta_gemv_t_stack(int n, int k, const double* M, const double* x,
                                                 const double* s, double* y) {
  const int tot = k * n;
  for (int o0 = threadIdx.x; o0 < tot; o0 += 4 * NT) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const double* col[4];
    bool on[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int o = o0 + u * NT;
      const int i = o < tot ? o / n : 0, c = o < tot ? o % n : 0;
      on[u] = o < tot && s[i] != 0.0;
      col[u] = M + (size_t)i * n * n + c;
    }
    for (int r = 0; r < n; ++r) {
      const double xr = x[r];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (on[u]) acc[u] = fma(col[u][(size_t)r * n], xr, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int o = o0 + u * NT;
      if (o < tot) y[o] = s[o / n] * acc[u];
    }
  }
  __syncthreads();
}

// y = s M^T x (+ y when accumulate), one thread per column; y must not alias x
__device__ __forceinline__ void cta_gemv_t(int n, const double* M, const double* x, double s,
                                           double* y, bool accumulate) {
  for (int c = threadIdx.x; c < n; c += NT) {
    double acc = 0.0;
    for (int r = 0; r < n; ++r) acc = fma(M[(size_t)r * n + c], x[r], acc);
    y[c] = accumulate ? fma(s, acc, y[c]) : s * acc;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// adjoint of the action (real, double, one vector): JOB_ADJ
//
// The factors of every I - c_i B serve 2N solves with one right-hand side
// each, so each processor forms its inverse once (Sec. 1: each processor
// computes an inverse; d column solves of its LU factors), and every step's
// solve is a CTA-wide matrix-vector product: Y_i = c_i M_i^-1 u forward,
// lambda_i = b_i M_i^-T wbar in reverse.
// ---------------------------------------------------------------------------
template <int NB>
__device__ __noinline__ void run_adjoint(const FmJob& J, const FmCoef& cf, int b, char* ws, char* smem) {
  using T = double;
  using TT = Tr<T>;
  const int tid = threadIdx.x;
  const int n = J.d[b];
  const int64_t off = J.off[b], vo = J.voff[b];
  const double t = J.t[b];
  const long long N = J.nsteps_dev[b];
  const int k = cf.k;
  const WsLayout L = ws_layout(JOB_ADJ, n, 1, k, 8, 8, J.nsteps_max);
  T* B = (T*)(ws + L.B);
  T* Cb = (T*)(ws + L.C);   // Bbar accumulator (n x n)
  T* u = (T*)(ws + L.U);
  T* ub = (T*)(ws + L.U2);
  T* wb = (T*)(ws + L.Wc);
  T* wbp = (T*)(ws + L.Wn);
  T* y = (T*)(ws + L.LUs);    // the reverse products' k n outputs (the factors
                              // are not used once the inverses are formed)
  T* Wst = (T*)(ws + L.Wst);
  T* Yst = (T*)(ws + L.Yst);
  const T* A = (const T*)J.A + off;
  int info = 0;
  if (N <= 0 || N > J.nsteps_max) info = -3;
  const double h = t / (double)(N > 0 ? N : 1);
  for (int e = tid; e < n * n; e += NT) {
    B[e] = TT::rscale(A[e], h);
    Cb[e] = 0.0;
  }
  __syncthreads();
  for (int i = 0; i < k && info == 0; ++i) {
    if (cf.c_re[i] == 0.0) continue;
    T* Ci = (T*)(ws + L.Cs) + (size_t)i * n * n;
    T* LUi = (T*)(ws + L.LUs) + (size_t)i * n * n;
    int* pivi = (int*)(ws + L.pivs) + (size_t)i * n;
    double* Di = (double*)(ws + L.Ds) + (size_t)i * n;
    build_shift<T, T>(n, cf.c_re[i], 0.0, B, Ci, LUi, Di, false);
    int fi = cta_getrf<T, NB>(n, LUi, n, pivi, (T*)smem);
    if (fi) info = i * n + fi;
  }
  // M_i^-1 in place of C_i (not used past the factorization)
  for (int i = 0; i < k && info == 0; ++i) {
    if (cf.c_re[i] == 0.0) continue;
    T* Inv = (T*)(ws + L.Cs) + (size_t)i * n * n;
    for (int e = tid; e < n * n; e += NT) Inv[e] = (e / n == e % n) ? 1.0 : 0.0;
    __syncthreads();
    cta_getrs<T, NB>(n, (T*)(ws + L.LUs) + (size_t)i * n * n, n, (int*)(ws + L.pivs) + (size_t)i * n,
                     n, Inv, n, (T*)smem);
  }
  if (info == 0) {
    // per-node scales: c_i for the forward products, b_i for the reverse ones
    // (0 for a zero node, whose inverse is not formed)
    double* sc = (double*)smem;  // 2 k doubles
    for (int i = tid; i < k; i += NT) {
      sc[i] = cf.c_re[i];
      sc[k + i] = cf.c_re[i] != 0.0 ? cf.b_re[0][i] : 0.0;
    }
    // forward sweep, storing w_q and Y_iq: u = B w, every Y_iq = c_i M_i^-1 u
    // in one stacked product, w_q = a0 w + sum_i b_i Y_iq (ascending i)
    for (int r = tid; r < n; r += NT) Wst[r] = ((const T*)J.V)[vo + r];
    __syncthreads();
    const T* Inv = (const T*)(ws + L.Cs);
    for (long long q = 1; q <= N; ++q) {
      const T* wp = Wst + (size_t)(q - 1) * n;
      T* wq = Wst + (size_t)q * n;
      T* yq = Yst + (size_t)(q - 1) * k * n;
      cta_gemv(n, B, wp, 1.0, u);
      cta_gemv_stack(n, k, Inv, u, sc, yq);
      for (int r = tid; r < n; r += NT) {
        T v = TT::rscale(wp[r], cf.a0[0]);
        for (int i = 0; i < k; ++i)
          if (cf.c_re[i] != 0.0) v = TT::add(v, TT::rscale(yq[(size_t)i * n + r], cf.b_re[0][i]));
        wq[r] = v;
      }
      __syncthreads();
    }
    for (int r = tid; r < n; r += NT) {
      ((T*)J.W)[vo + r] = Wst[(size_t)N * n + r];
      wb[r] = J.wbar[vo + r];
    }
    __syncthreads();
    // reverse sweep: lambda_i = b_i M_i^-T wbar (one stacked product),
    // ubar = sum_i c_i lambda_i, wbar_{q-1} = a0 wbar + B^T ubar; the terms
    // of Bbar = sum_q (sum_i c_i lambda_iq Y_iq^T + ubar_q w_{q-1}^T) are kept
    // (c_i lambda_iq as column (q-1) k + i of LamY, ubar_q as column q-1 of UB)
    // and summed by two products after the sweep
    T* LamY = (T*)(ws + L.LamY);
    T* UB = (T*)(ws + L.UB);
    const size_t ldl = (size_t)k * N;
    for (long long q = N; q >= 1; --q) {
      cta_gemv_t_stack(n, k, Inv, wb, sc + k, y);
      for (int r = tid; r < n; r += NT) {
        T ubr = 0.0;
        for (int i = 0; i < k; ++i) {
          const double c = cf.c_re[i];
          const T l = c != 0.0 ? TT::rscale(y[(size_t)i * n + r], c) : 0.0;
          LamY[(size_t)r * ldl + (size_t)(q - 1) * k + i] = l;
          ubr = TT::add(ubr, l);
        }
        ub[r] = ubr;
        UB[(size_t)r * N + (q - 1)] = ubr;
        wbp[r] = TT::rscale(wb[r], cf.a0[0]);
      }
      __syncthreads();
      cta_gemv_t(n, B, ub, 1.0, wbp, true);
      for (int r = tid; r < n; r += NT) wb[r] = wbp[r];
      __syncthreads();
    }
    // Bbar = LamY Yst + UB Wst (rows 0..N-1 of Wst are w_0 .. w_{N-1})
    cta_gemm<T>(n, n, (int)(k * N), 1.0, LamY, (int)ldl, Yst, n, 0.0, Cb, n, (T*)(smem + 256));
    cta_gemm<T>(n, n, (int)N, 1.0, UB, (int)N, Wst, n, 1.0, Cb, n, (T*)(smem + 256));
    for (int e = tid; e < n * n; e += NT) J.Abar[off + e] = TT::rscale(Cb[e], h);
    for (int r = tid; r < n; r += NT) J.vbar[vo + r] = wb[r];
  }
  if (tid == 0 && J.info) J.info[b] = info;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// the persistent kernel: a work queue over matrices, largest first
// ---------------------------------------------------------------------------
// Two CTAs share an SM on the double path (more warps to feed the FP64
// pipe); the tensor-core path keeps one CTA per SM (its operand staging and
// tensor memory are sized for the whole SM).
template <class T, class TL, int NB, bool TCK = false>
__global__ void __launch_bounds__(NT, TCK ? 1 : 2) fm_persistent(FmJob J, FmCoef cf) {
  extern __shared__ __align__(1024) char smem[];
  __shared__ int s_item;
  __shared__ oz::Ctx s_oz;
  __shared__ __align__(8) uint64_t s_bars[4];
  __shared__ uint32_t s_tmem;
  // the shifted systems of the coefficient set (filled per matrix by one thread),
  // then base[2] and the system count
  __shared__ __align__(16) Sys s_plan[kMaxTerms + 1];
  char* ws = J.ws + (size_t)blockIdx.x * J.ws_stride;
  const int limit = J.order ? *(volatile int*)(J.counter + 1) : J.batch;
  oz::Ctx* oc = nullptr;
  if constexpr (TCK) {
    // mbarriers for the split products; tensor memory is taken per product
    if (threadIdx.x == 0) {
      for (int i = 0; i < 4; ++i) tc::mbar_init(&s_bars[i], 1);
      tc::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_oz.tslot = &s_tmem;
      s_oz.tmem = 0;
      s_oz.bar = s_bars;
      s_oz.smem = (unsigned char*)(((uintptr_t)smem + 1023) & ~(uintptr_t)1023);
      s_oz.use[0] = s_oz.use[1] = 0;
      s_oz.err = 0;
    }
    __syncthreads();
    oc = &s_oz;
  }
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(J.counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= limit) break;
    if constexpr (TCK) {
      if (s_oz.err) break;  // a tensor-core wait timed out: stop taking work
    }
    const int b = J.order ? J.order[item] : item;
    if (J.kind == JOB_EXPM || J.kind == JOB_PHI1 || J.kind == JOB_PHI1MV || J.kind == JOB_TRIG)
      run_matfun<T, TL, NB>(J, cf, b, ws, smem + 1024, oc, s_plan);
    else if (J.kind == JOB_EXPMV)
      run_action<T, TL, NB>(J, cf, b, ws, smem + 1024, oc, s_plan);
    else if constexpr (sizeof(T) == 8 && sizeof(TL) == 8)
      run_adjoint<NB>(J, cf, b, ws, smem + 1024);
  }
}

// dynamic shared memory the kernel needs for matrices up to n
template <class T, int NB>
inline size_t fm_smem_bytes(int n, bool tck = false) {
  size_t getrf = ((size_t)n * NB + 2 * GK * GLD) * sizeof(T) + 256;
  size_t getrs = ((size_t)NB * NB + 2 * GK * GLD) * sizeof(T);
  size_t gemm = 256 + 2 * GK * GLD * sizeof(T);
  // left-looking solves: a 16 x n panel and the partial sums
  size_t slice = ((size_t)16 * n + (size_t)NT * 16 + 64) * sizeof(T);
  if (slice > 200 * 1024) slice = 200 * 1024;
  size_t m = getrf > getrs ? getrf : getrs;
  m = m > gemm ? m : gemm;
  m = m > slice ? m : slice;
  size_t need = 1024 + m + 512;
  if (tck && need < oz::SMEM + 2048) need = oz::SMEM + 2048;
  return need;
}

}  // namespace fmk
