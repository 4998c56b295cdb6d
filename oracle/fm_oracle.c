/*
 * fm_oracle.c -- plain, slow, FP64 CPU oracle for the method of
 * S. Blanes, "Parallel computation of functions of matrices and their action
 * on vectors" (arXiv:2210.03714).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of bench.py may load this library.  It shares no code with the CUDA
 * library: it has its own types, its own LU, its own everything.
 *
 * What it computes, step by step, in the paper's order:
 *   1. eta = ||tA||_1 (or a caller bound), Sec. 1 "scaling" and Sec. 5;
 *   2. s = max(0, ceil(log2(eta/theta))), B = tA/2^s (Sec. 1: N = 2^s so that
 *      ||A/N|| < theta, theta from the forward bound of Sec. 3);
 *   3. for every term with c_i != 0: textbook LU with partial pivoting of
 *      M_i = I - c_i B (Sec. 1: "LU decomposition and d triangular solves"),
 *      then Y_i = M_i^{-1} (c_i B R) (roundoff form, Eq. ParallRoundOff;
 *      action form, Eq. Frac10R: the product B R is formed once);
 *   4. r(B) R = a0 R + d1 B R + d2 B^2 R + sum_i b_i Y_i  (ascending i);
 *      the plain form (Eq. rat1 / ParallHybrid) solves with RHS R instead and
 *      uses d0 = a0 - sum_i b_i;
 *   5. s squarings F <- F F (Sec. 1); for phi_1 the doubling
 *      phi1(2X) = (e^X + I) phi1(X) / 2 (Sec. 1; the printed version carries a
 *      stray factor t, this is the identity that holds); for the action,
 *      N = ceil(eta/theta) steps v_n = r(B) v_{n-1}, B = tA/N, the LU factors
 *      computed once (Sec. 4.4 remarks: the factorization is done only once).
 *   6. the adjoint (reverse sweep) of that discrete action map.
 *
 * Layout: row-major, dense, leading dimension = number of columns.
 * Every loop is written in the order of the textbook definition; there is
 * no blocking.  Compile with -ffp-contract=off so every operation rounds as
 * written.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int k;                 /* number of terms (c = 0 terms included)           */
  const double *c_re, *c_im, *b_re, *b_im;
  int conj_pair;         /* 1: each term stands for 2 Re(b_i / (1 - c_i x))   */
  double a0, d1, d2;     /* a0 = r(0); d1, d2: hybrid polynomial part         */
  double theta;          /* ||B|| bound for the tolerance                     */
} orc_coeffs;

enum { ORC_ROUNDOFF = 0, ORC_PLAIN = 1 };

/* ------------------------------------------------------------------------ */
/* basic dense helpers                                                       */
/* ------------------------------------------------------------------------ */

/* ||A||_1 = max_j sum_i |a_ij| */
double orc_norm1(int n, const double* A) {
  double best = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += fabs(A[(size_t)i * n + j]);
    if (s > best || isnan(s)) best = s;
  }
  return best;
}

double orc_znorm1(int n, const double complex* A) {
  double best = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += cabs(A[(size_t)i * n + j]);
    if (s > best || isnan(s)) best = s;
  }
  return best;
}

/* smallest s >= 0 with eta / 2^s <= theta (Sec. 1, N = 2^s) */
int orc_select_s(double eta, double theta) {
  int s = 0;
  while (eta > ldexp(theta, s) && s < 1023) ++s;
  return s;
}

/* smallest N >= 1 with eta / N <= theta (action recurrence, Sec. 1) */
long orc_select_nsteps(double eta, double theta) {
  double q = ceil(eta / theta);
  return q < 1.0 ? 1 : (long)q;
}

/* C (n x m) = A (n x p) * B (p x m) */
static void matmul(int n, int p, int m, const double* A, const double* B, double* C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int l = 0; l < p; ++l) s += A[(size_t)i * p + l] * B[(size_t)l * m + j];
      C[(size_t)i * m + j] = s;
    }
}

static void zmatmul(int n, int p, int m, const double complex* A, const double complex* B,
                    double complex* C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double complex s = 0.0;
      for (int l = 0; l < p; ++l) s += A[(size_t)i * p + l] * B[(size_t)l * m + j];
      C[(size_t)i * m + j] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* textbook Gaussian elimination with partial pivoting (outer-product form) */
/* ------------------------------------------------------------------------ */

/* In place: A = P^T L U; piv[k] = row swapped with k at step k.  Ties in the
 * pivot search go to the lowest row index.  Returns 0, or j+1 when the pivot
 * of column j is exactly zero (the factorization stops there). */
int orc_gepp(int n, double* A, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = fabs(A[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)p * n + j];
        A[(size_t)p * n + j] = t;
      }
    double pv = A[(size_t)k * n + k];
    if (pv == 0.0) return k + 1;
    for (int i = k + 1; i < n; ++i) A[(size_t)i * n + k] /= pv;
    for (int i = k + 1; i < n; ++i) {
      double l = A[(size_t)i * n + k];
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return 0;
}

/* Solve (P^T L U) X = X_in for m right-hand sides, X is n x m, in place. */
void orc_getrs(int n, const double* LU, const int* piv, int m, double* X) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k)
      for (int j = 0; j < m; ++j) {
        double t = X[(size_t)k * m + j];
        X[(size_t)k * m + j] = X[(size_t)piv[k] * m + j];
        X[(size_t)piv[k] * m + j] = t;
      }
  for (int i = 0; i < n; ++i)           /* forward: unit lower L */
    for (int l = 0; l < i; ++l) {
      double f = LU[(size_t)i * n + l];
      for (int j = 0; j < m; ++j) X[(size_t)i * m + j] -= f * X[(size_t)l * m + j];
    }
  for (int i = n - 1; i >= 0; --i) {    /* backward: upper U */
    for (int l = i + 1; l < n; ++l) {
      double f = LU[(size_t)i * n + l];
      for (int j = 0; j < m; ++j) X[(size_t)i * m + j] -= f * X[(size_t)l * m + j];
    }
    double d = LU[(size_t)i * n + i];
    for (int j = 0; j < m; ++j) X[(size_t)i * m + j] /= d;
  }
}

/* Solve (P^T L U)^T X = X_in (used by the adjoint). */
void orc_getrs_trans(int n, const double* LU, const int* piv, int m, double* X) {
  /* U^T z = x (forward), L^T w = z (backward), then undo the swaps */
  for (int i = 0; i < n; ++i) {
    for (int l = 0; l < i; ++l) {
      double f = LU[(size_t)l * n + i];
      for (int j = 0; j < m; ++j) X[(size_t)i * m + j] -= f * X[(size_t)l * m + j];
    }
    double d = LU[(size_t)i * n + i];
    for (int j = 0; j < m; ++j) X[(size_t)i * m + j] /= d;
  }
  for (int i = n - 1; i >= 0; --i)
    for (int l = i + 1; l < n; ++l) {
      double f = LU[(size_t)l * n + i];
      for (int j = 0; j < m; ++j) X[(size_t)i * m + j] -= f * X[(size_t)l * m + j];
    }
  for (int k = n - 1; k >= 0; --k)
    if (piv[k] != k)
      for (int j = 0; j < m; ++j) {
        double t = X[(size_t)k * m + j];
        X[(size_t)k * m + j] = X[(size_t)piv[k] * m + j];
        X[(size_t)piv[k] * m + j] = t;
      }
}

int orc_zgepp(int n, double complex* A, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = cabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = cabs(A[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        double complex t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)p * n + j];
        A[(size_t)p * n + j] = t;
      }
    double complex pv = A[(size_t)k * n + k];
    if (pv == 0.0) return k + 1;
    for (int i = k + 1; i < n; ++i) A[(size_t)i * n + k] /= pv;
    for (int i = k + 1; i < n; ++i) {
      double complex l = A[(size_t)i * n + k];
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return 0;
}

void orc_zgetrs(int n, const double complex* LU, const int* piv, int m, double complex* X) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k)
      for (int j = 0; j < m; ++j) {
        double complex t = X[(size_t)k * m + j];
        X[(size_t)k * m + j] = X[(size_t)piv[k] * m + j];
        X[(size_t)piv[k] * m + j] = t;
      }
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < i; ++l) {
      double complex f = LU[(size_t)i * n + l];
      for (int j = 0; j < m; ++j) X[(size_t)i * m + j] -= f * X[(size_t)l * m + j];
    }
  for (int i = n - 1; i >= 0; --i) {
    for (int l = i + 1; l < n; ++l) {
      double complex f = LU[(size_t)i * n + l];
      for (int j = 0; j < m; ++j) X[(size_t)i * m + j] -= f * X[(size_t)l * m + j];
    }
    double complex d = LU[(size_t)i * n + i];
    for (int j = 0; j < m; ++j) X[(size_t)i * m + j] /= d;
  }
}

/* ------------------------------------------------------------------------ */
/* the rational approximant applied to a block R (Sec. 2, Eq. ParallRoundOff) */
/* ------------------------------------------------------------------------ */

static int all_finite(size_t n, const double* x) {
  for (size_t i = 0; i < n; ++i)
    if (!isfinite(x[i])) return 0;
  return 1;
}

/* Factorizations of M_i = I - c_i B for a real set (c_i real, c_i != 0).
 * lu: k blocks of n*n, piv: k blocks of n.  Returns info (0 or shift*n+col). */
static int factor_real(int n, const double* B, const orc_coeffs* cs, double* lu, int* piv) {
  for (int i = 0; i < cs->k; ++i) {
    double c = cs->c_re[i];
    if (c == 0.0) continue;
    double* M = lu + (size_t)i * n * n;
    for (int r = 0; r < n; ++r)
      for (int q = 0; q < n; ++q)
        M[(size_t)r * n + q] = (r == q ? 1.0 : 0.0) - c * B[(size_t)r * n + q];
    int info = orc_gepp(n, M, piv + (size_t)i * n);
    if (info) return i * n + info;
  }
  return 0;
}

/* r(B) R for several real coefficient sets sharing the same c_i (Sec. 2:
 * different functions from the same resolvents only need new b_i).
 * R = NULL means R = I (m = n).  lu/piv from factor_real.  outs[j] is n x m. */
static void apply_real(int n, const double* B, int nsets, const orc_coeffs* const* sets,
                       int form, int m, const double* R, const double* lu, const int* piv,
                       double* const* outs) {
  const orc_coeffs* c0 = sets[0];
  size_t nm = (size_t)n * m;
  double* Rm = malloc(nm * sizeof(double));
  double* U = malloc(nm * sizeof(double));
  double* U2 = malloc(nm * sizeof(double));
  double* Y = malloc(nm * sizeof(double));
  if (R) memcpy(Rm, R, nm * sizeof(double));
  else for (int r = 0; r < n; ++r) for (int q = 0; q < n; ++q) Rm[(size_t)r * n + q] = (r == q);
  /* U = B R (the single product of Eq. Frac10R); for R = I this equals B */
  if (R) matmul(n, n, m, B, Rm, U); else memcpy(U, B, nm * sizeof(double));
  int need_b2 = 0;
  for (int j = 0; j < nsets; ++j) need_b2 |= (sets[j]->d2 != 0.0);
  if (need_b2) matmul(n, n, m, B, U, U2);
  for (int j = 0; j < nsets; ++j) {
    const orc_coeffs* cs = sets[j];
    double base = cs->a0;
    if (form == ORC_PLAIN) for (int i = 0; i < cs->k; ++i) base -= cs->b_re[i];
    for (size_t e = 0; e < nm; ++e) outs[j][e] = base * Rm[e];
    if (cs->d1 != 0.0) for (size_t e = 0; e < nm; ++e) outs[j][e] += cs->d1 * U[e];
    if (cs->d2 != 0.0) for (size_t e = 0; e < nm; ++e) outs[j][e] += cs->d2 * U2[e];
  }
  for (int i = 0; i < c0->k; ++i) {
    double c = c0->c_re[i];
    if (c == 0.0) {
      /* roundoff form: c_i x / (1 - c_i x) = 0; plain form: b_i * I */
      if (form == ORC_PLAIN)
        for (int j = 0; j < nsets; ++j)
          for (size_t e = 0; e < nm; ++e) outs[j][e] += sets[j]->b_re[i] * Rm[e];
      continue;
    }
    if (form == ORC_ROUNDOFF) for (size_t e = 0; e < nm; ++e) Y[e] = c * U[e];
    else memcpy(Y, Rm, nm * sizeof(double));
    orc_getrs(n, lu + (size_t)i * n * n, piv + (size_t)i * n, m, Y);
    for (int j = 0; j < nsets; ++j) {
      double b = sets[j]->b_re[i];
      for (size_t e = 0; e < nm; ++e) outs[j][e] += b * Y[e];
    }
  }
  free(Rm); free(U); free(U2); free(Y);
}

/* Conjugate-pair sets on a real B (Eq. Pade4 / Pade4phi1): each term is
 * 2 Re(b_i Y_i) with complex Y_i = (I - c_i B)^{-1} (c_i B R). */
static int apply_conj(int n, const double* B, int nsets, const orc_coeffs* const* sets,
                      int form, int m, const double* R, double* const* outs) {
  const orc_coeffs* c0 = sets[0];
  size_t nm = (size_t)n * m, nn = (size_t)n * n;
  double* Rm = malloc(nm * sizeof(double));
  double* U = malloc(nm * sizeof(double));
  double complex* M = malloc(nn * sizeof(double complex));
  double complex* Y = malloc(nm * sizeof(double complex));
  int* piv = malloc((size_t)n * sizeof(int));
  int info = 0;
  if (R) memcpy(Rm, R, nm * sizeof(double));
  else for (int r = 0; r < n; ++r) for (int q = 0; q < n; ++q) Rm[(size_t)r * n + q] = (r == q);
  if (R) matmul(n, n, m, B, Rm, U); else memcpy(U, B, nm * sizeof(double));
  for (int j = 0; j < nsets; ++j) {
    const orc_coeffs* cs = sets[j];
    double base = cs->a0;
    if (form == ORC_PLAIN) for (int i = 0; i < cs->k; ++i) base -= 2.0 * cs->b_re[i];
    for (size_t e = 0; e < nm; ++e) outs[j][e] = base * Rm[e];
  }
  for (int i = 0; i < c0->k && !info; ++i) {
    double complex c = c0->c_re[i] + I * c0->c_im[i];
    for (int r = 0; r < n; ++r)
      for (int q = 0; q < n; ++q)
        M[(size_t)r * n + q] = (r == q ? 1.0 : 0.0) - c * B[(size_t)r * n + q];
    int f = orc_zgepp(n, M, piv);
    if (f) { info = i * n + f; break; }
    for (size_t e = 0; e < nm; ++e) Y[e] = (form == ORC_ROUNDOFF) ? c * U[e] : Rm[e];
    orc_zgetrs(n, M, piv, m, Y);
    for (int j = 0; j < nsets; ++j) {
      double complex b = sets[j]->b_re[i] + I * sets[j]->b_im[i];
      for (size_t e = 0; e < nm; ++e) outs[j][e] += 2.0 * creal(b * Y[e]);
    }
  }
  free(Rm); free(U); free(M); free(Y); free(piv);
  return info;
}

/* r(B) R for one or more sets (shared c).  Returns info. */
int orc_rational_apply(int n, const double* B, int nsets, const orc_coeffs* const* sets,
                       int form, int m, const double* R, double* const* outs) {
  if (sets[0]->conj_pair) return apply_conj(n, B, nsets, sets, form, m, R, outs);
  double* lu = malloc((size_t)sets[0]->k * n * n * sizeof(double));
  int* piv = malloc((size_t)sets[0]->k * n * sizeof(int));
  int info = factor_real(n, B, sets[0], lu, piv);
  if (!info) apply_real(n, B, nsets, sets, form, m, R, lu, piv, outs);
  free(lu); free(piv);
  return info;
}

/* ------------------------------------------------------------------------ */
/* scaling and squaring: exp(tA) (Sec. 1)                                    */
/* ------------------------------------------------------------------------ */

/* F = r(B)^(2^s), B = tA/2^s.  anorm > 0 replaces ||tA||_1 by anorm*|t|.
 * s_fixed >= 0 forces s.  Returns info; *s_out receives s. */
int orc_expm(int n, const double* A, double t, const orc_coeffs* cs, int form, double anorm,
             int s_fixed, double* F, int* s_out) {
  size_t nn = (size_t)n * n;
  if (!all_finite(nn, A) || !isfinite(t)) return -2;
  double* B = malloc(nn * sizeof(double));
  double* T = malloc(nn * sizeof(double));
  for (size_t e = 0; e < nn; ++e) B[e] = t * A[e];
  double eta = anorm > 0.0 ? anorm * fabs(t) : orc_norm1(n, B);
  int s = s_fixed >= 0 ? s_fixed : orc_select_s(eta, cs->theta);
  for (size_t e = 0; e < nn; ++e) B[e] = ldexp(B[e], -s);
  const orc_coeffs* sets[1] = {cs};
  double* outs[1] = {F};
  int info = orc_rational_apply(n, B, 1, sets, form, n, NULL, outs);
  for (int q = 0; q < s && !info; ++q) {
    matmul(n, n, n, F, F, T);
    memcpy(F, T, nn * sizeof(double));
  }
  if (s_out) *s_out = s;
  free(B); free(T);
  return info;
}

/* phi1(tA) (and exp(tA)) by the doubling phi1(2X) = (e^X + I) phi1(X) / 2,
 * with E and Phi from the same resolvents.  theta = min of the two sets. */
int orc_phi1(int n, const double* A, double t, const orc_coeffs* ce, const orc_coeffs* cp,
             int form, double anorm, int s_fixed, double* Phi, double* E, int* s_out) {
  size_t nn = (size_t)n * n;
  if (!all_finite(nn, A) || !isfinite(t)) return -2;
  double* B = malloc(nn * sizeof(double));
  double* Eb = malloc(nn * sizeof(double));
  double* T = malloc(nn * sizeof(double));
  for (size_t e = 0; e < nn; ++e) B[e] = t * A[e];
  double eta = anorm > 0.0 ? anorm * fabs(t) : orc_norm1(n, B);
  double th = ce->theta < cp->theta ? ce->theta : cp->theta;
  int s = s_fixed >= 0 ? s_fixed : orc_select_s(eta, th);
  for (size_t e = 0; e < nn; ++e) B[e] = ldexp(B[e], -s);
  const orc_coeffs* sets[2] = {ce, cp};
  double* outs[2] = {Eb, Phi};
  int info = orc_rational_apply(n, B, 2, sets, form, n, NULL, outs);
  for (int q = 0; q < s && !info; ++q) {
    /* Phi <- (E + I) Phi / 2, then E <- E E */
    for (int r = 0; r < n; ++r) Eb[(size_t)r * n + r] += 1.0;
    matmul(n, n, n, Eb, Phi, T);
    for (size_t e = 0; e < nn; ++e) Phi[e] = 0.5 * T[e];
    for (int r = 0; r < n; ++r) Eb[(size_t)r * n + r] -= 1.0;
    matmul(n, n, n, Eb, Eb, T);
    memcpy(Eb, T, nn * sizeof(double));
  }
  if (E) memcpy(E, Eb, nn * sizeof(double));
  if (s_out) *s_out = s;
  free(B); free(Eb); free(T);
  return info;
}

/* cos(tA) and sin(tA) from one set of resolvents: the two sets share the c_i
 * (Sec. 2: another function from the same F_i only needs new b_i), scaling
 * B = tA/2^s, then s steps of the double-angle formulae of Sec. 1,
 * cos(2X) = 2 cos(X)^2 - I and sin(2X) = 2 sin(X) cos(X).
 * theta = min of the two sets. */
int orc_trig(int n, const double* A, double t, const orc_coeffs* cc, const orc_coeffs* cs,
             int form, double anorm, int s_fixed, double* C, double* S, int* s_out) {
  size_t nn = (size_t)n * n;
  if (!all_finite(nn, A) || !isfinite(t)) return -2;
  double* B = malloc(nn * sizeof(double));
  double* T = malloc(nn * sizeof(double));
  double* T2 = malloc(nn * sizeof(double));
  for (size_t e = 0; e < nn; ++e) B[e] = t * A[e];
  double eta = anorm > 0.0 ? anorm * fabs(t) : orc_norm1(n, B);
  double th = cc->theta < cs->theta ? cc->theta : cs->theta;
  int s = s_fixed >= 0 ? s_fixed : orc_select_s(eta, th);
  for (size_t e = 0; e < nn; ++e) B[e] = ldexp(B[e], -s);
  const orc_coeffs* sets[2] = {cc, cs};
  double* outs[2] = {C, S};
  int info = orc_rational_apply(n, B, 2, sets, form, n, NULL, outs);
  for (int q = 0; q < s && !info; ++q) {
    matmul(n, n, n, S, C, T);   /* sin(X) cos(X) */
    matmul(n, n, n, C, C, T2);  /* cos(X)^2 */
    for (size_t e = 0; e < nn; ++e) {
      S[e] = 2.0 * T[e];
      C[e] = 2.0 * T2[e];
    }
    for (int r = 0; r < n; ++r) C[(size_t)r * n + r] -= 1.0;
  }
  if (s_out) *s_out = s;
  free(B); free(T); free(T2);
  return info;
}

/* r(tA) for one set, with no range reduction: B = tA and r(B) as Sec. 2
 * defines it (f(B) ~ r(B) for sufficiently small ||B||; e.g. the weights for
 * log(1 - x) printed after Eq. Frac4bi0, for which the paper gives no scaling). */
int orc_rfun(int n, const double* A, double t, const orc_coeffs* cs, int form, double* F) {
  size_t nn = (size_t)n * n;
  if (!all_finite(nn, A) || !isfinite(t)) return -2;
  double* B = malloc(nn * sizeof(double));
  for (size_t e = 0; e < nn; ++e) B[e] = t * A[e];
  const orc_coeffs* sets[1] = {cs};
  double* outs[1] = {F};
  int info = orc_rational_apply(n, B, 1, sets, form, n, NULL, outs);
  free(B);
  return info;
}

/* ------------------------------------------------------------------------ */
/* action: exp(tA) V by N steps of r(tA/N) with the LU reused (Sec. 1, 2, 5) */
/* ------------------------------------------------------------------------ */

int orc_expmv(int n, const double* A, double t, const orc_coeffs* cs, int form, double anorm,
              long nsteps, int m, const double* V, double* W, long* n_out) {
  size_t nn = (size_t)n * n, nm = (size_t)n * m;
  if (!all_finite(nn, A) || !all_finite(nm, V) || !isfinite(t)) return -2;
  double* B = malloc(nn * sizeof(double));
  double* Wn = malloc(nm * sizeof(double));
  for (size_t e = 0; e < nn; ++e) B[e] = t * A[e];
  double eta = anorm > 0.0 ? anorm * fabs(t) : orc_norm1(n, B);
  long N = nsteps > 0 ? nsteps : orc_select_nsteps(eta, cs->theta);
  double h = t / (double)N;
  for (size_t e = 0; e < nn; ++e) B[e] = h * A[e];
  memcpy(W, V, nm * sizeof(double));
  const orc_coeffs* sets[1] = {cs};
  double* outs[1] = {Wn};
  int info = 0;
  if (cs->conj_pair) {
    for (long q = 0; q < N && !info; ++q) {
      info = apply_conj(n, B, 1, sets, form, m, W, outs);
      memcpy(W, Wn, nm * sizeof(double));
    }
  } else {
    double* lu = malloc((size_t)cs->k * nn * sizeof(double));
    int* piv = malloc((size_t)cs->k * n * sizeof(int));
    info = factor_real(n, B, cs, lu, piv);
    for (long q = 0; q < N && !info; ++q) {
      apply_real(n, B, 1, sets, form, m, W, lu, piv, outs);
      memcpy(W, Wn, nm * sizeof(double));
    }
    free(lu); free(piv);
  }
  if (n_out) *n_out = N;
  free(B); free(Wn);
  return info;
}

/* phi1(tA) V through the matrix phi1 (doubling) and one product. */
int orc_phi1mv(int n, const double* A, double t, const orc_coeffs* ce, const orc_coeffs* cp,
               int form, double anorm, int m, const double* V, double* W, int* s_out) {
  size_t nn = (size_t)n * n;
  double* Phi = malloc(nn * sizeof(double));
  int info = orc_phi1(n, A, t, ce, cp, form, anorm, -1, Phi, NULL, s_out);
  if (!info) matmul(n, n, m, Phi, V, W);
  free(Phi);
  return info;
}

/* ------------------------------------------------------------------------ */
/* adjoint of the discrete action map (roundoff form, real, c_i real)        */
/* ------------------------------------------------------------------------ */

/* Forward: w_0 = v; u_q = B w_{q-1}; Y_iq = M_i^{-1}(c_i u_q);
 *          w_q = a0 w_{q-1} + sum_i b_i Y_iq  (q = 1..N), B = hA, h = t/N.
 * Given wbar = dL/dw_N, returns Abar = dL/dA (n x n) and vbar = dL/dv (n),
 * for fixed N (the step count is not differentiated).  m = 1 vector. */
int orc_expmv_adjoint(int n, const double* A, double t, const orc_coeffs* cs, long N,
                      const double* v, const double* wbar_in, double* Abar, double* vbar) {
  size_t nn = (size_t)n * n;
  int K = cs->k;
  double h = t / (double)N;
  double* B = malloc(nn * sizeof(double));
  for (size_t e = 0; e < nn; ++e) B[e] = h * A[e];
  double* lu = malloc((size_t)K * nn * sizeof(double));
  int* piv = malloc((size_t)K * n * sizeof(int));
  int info = factor_real(n, B, cs, lu, piv);
  if (info) { free(B); free(lu); free(piv); return info; }
  /* forward sweep, storing w_q (q = 0..N) and Y_iq */
  double* w = malloc((size_t)(N + 1) * n * sizeof(double));
  double* Y = malloc((size_t)N * K * n * sizeof(double));
  double* u = malloc((size_t)n * sizeof(double));
  memcpy(w, v, (size_t)n * sizeof(double));
  for (long q = 1; q <= N; ++q) {
    const double* wp = w + (size_t)(q - 1) * n;
    double* wq = w + (size_t)q * n;
    matmul(n, n, 1, B, wp, u);
    for (int r = 0; r < n; ++r) wq[r] = cs->a0 * wp[r];
    for (int i = 0; i < K; ++i) {
      double c = cs->c_re[i];
      double* y = Y + ((size_t)(q - 1) * K + i) * n;
      if (c == 0.0) { memset(y, 0, (size_t)n * sizeof(double)); continue; }
      for (int r = 0; r < n; ++r) y[r] = c * u[r];
      orc_getrs(n, lu + (size_t)i * nn, piv + (size_t)i * n, 1, y);
      for (int r = 0; r < n; ++r) wq[r] += cs->b_re[i] * y[r];
    }
  }
  /* reverse sweep */
  double* wb = malloc((size_t)n * sizeof(double));
  double* wbp = malloc((size_t)n * sizeof(double));
  double* ub = malloc((size_t)n * sizeof(double));
  double* lam = malloc((size_t)n * sizeof(double));
  double* Bb = calloc(nn, sizeof(double));
  memcpy(wb, wbar_in, (size_t)n * sizeof(double));
  for (long q = N; q >= 1; --q) {
    const double* wp = w + (size_t)(q - 1) * n;
    for (int r = 0; r < n; ++r) { wbp[r] = cs->a0 * wb[r]; ub[r] = 0.0; }
    for (int i = 0; i < K; ++i) {
      double c = cs->c_re[i];
      if (c == 0.0) continue;
      const double* y = Y + ((size_t)(q - 1) * K + i) * n;
      /* Y = M^{-1} (c u): lam = M^{-T} (b_i wbar); ubar += c lam;
       * Mbar = -lam Y^T and M = I - c B give Bbar += c lam Y^T */
      for (int r = 0; r < n; ++r) lam[r] = cs->b_re[i] * wb[r];
      orc_getrs_trans(n, lu + (size_t)i * nn, piv + (size_t)i * n, 1, lam);
      for (int r = 0; r < n; ++r) ub[r] += c * lam[r];
      for (int r = 0; r < n; ++r)
        for (int s2 = 0; s2 < n; ++s2) Bb[(size_t)r * n + s2] += c * lam[r] * y[s2];
    }
    /* u = B w_{q-1}: Bbar += ubar w^T, wbar_{q-1} += B^T ubar */
    for (int r = 0; r < n; ++r)
      for (int s2 = 0; s2 < n; ++s2) Bb[(size_t)r * n + s2] += ub[r] * wp[s2];
    for (int s2 = 0; s2 < n; ++s2) {
      double acc = 0.0;
      for (int r = 0; r < n; ++r) acc += B[(size_t)r * n + s2] * ub[r];
      wbp[s2] += acc;
    }
    memcpy(wb, wbp, (size_t)n * sizeof(double));
  }
  for (size_t e = 0; e < nn; ++e) Abar[e] = h * Bb[e];
  memcpy(vbar, wb, (size_t)n * sizeof(double));
  free(B); free(lu); free(piv); free(w); free(Y); free(u);
  free(wb); free(wbp); free(ub); free(lam); free(Bb);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* complex matrices (z-variants): the same steps with complex c_i, b_i        */
/* ------------------------------------------------------------------------ */

/* Factorizations of M_i = I - c_i B for complex B, c_i (c_i != 0), as
 * factor_real does for real sets.  lu: k blocks of n*n, piv: k blocks of n.
 * Returns info (0 or shift*n+col). */
static int zfactor(int n, const double complex* B, const orc_coeffs* cs, double complex* lu,
                   int* piv) {
  for (int i = 0; i < cs->k; ++i) {
    double complex c = cs->c_re[i] + I * cs->c_im[i];
    if (c == 0.0) continue;
    double complex* M = lu + (size_t)i * n * n;
    for (int r = 0; r < n; ++r)
      for (int q = 0; q < n; ++q)
        M[(size_t)r * n + q] = (r == q ? 1.0 : 0.0) - c * B[(size_t)r * n + q];
    int f = orc_zgepp(n, M, piv + (size_t)i * n);
    if (f) return i * n + f;
  }
  return 0;
}

/* r(B) R with complex B, c, b and the factors from zfactor; R = NULL means I. */
static void zapply_lu(int n, const double complex* B, const orc_coeffs* cs, int form, int m,
                      const double complex* R, const double complex* lu, const int* piv,
                      double complex* out) {
  size_t nm = (size_t)n * m;
  double complex* Rm = malloc(nm * sizeof(double complex));
  double complex* U = malloc(nm * sizeof(double complex));
  double complex* U2 = malloc(nm * sizeof(double complex));
  double complex* Y = malloc(nm * sizeof(double complex));
  if (R) memcpy(Rm, R, nm * sizeof(double complex));
  else for (int r = 0; r < n; ++r) for (int q = 0; q < n; ++q) Rm[(size_t)r * n + q] = (r == q);
  if (R) zmatmul(n, n, m, B, Rm, U); else memcpy(U, B, nm * sizeof(double complex));
  if (cs->d2 != 0.0) zmatmul(n, n, m, B, U, U2);
  double complex base = cs->a0;
  if (form == ORC_PLAIN) for (int i = 0; i < cs->k; ++i) base -= cs->b_re[i] + I * cs->b_im[i];
  for (size_t e = 0; e < nm; ++e) out[e] = base * Rm[e];
  if (cs->d1 != 0.0) for (size_t e = 0; e < nm; ++e) out[e] += cs->d1 * U[e];
  if (cs->d2 != 0.0) for (size_t e = 0; e < nm; ++e) out[e] += cs->d2 * U2[e];
  for (int i = 0; i < cs->k; ++i) {
    double complex c = cs->c_re[i] + I * cs->c_im[i];
    double complex b = cs->b_re[i] + I * cs->b_im[i];
    if (c == 0.0) {
      if (form == ORC_PLAIN) for (size_t e = 0; e < nm; ++e) out[e] += b * Rm[e];
      continue;
    }
    for (size_t e = 0; e < nm; ++e) Y[e] = (form == ORC_ROUNDOFF) ? c * U[e] : Rm[e];
    orc_zgetrs(n, lu + (size_t)i * n * n, piv + (size_t)i * n, m, Y);
    for (size_t e = 0; e < nm; ++e) out[e] += b * Y[e];
  }
  free(Rm); free(U); free(U2); free(Y);
}

/* r(B) R with complex B, c, b; R = NULL means I.  Returns info. */
static int zapply(int n, const double complex* B, const orc_coeffs* cs, int form, int m,
                  const double complex* R, double complex* out) {
  double complex* lu = malloc((size_t)cs->k * n * n * sizeof(double complex));
  int* piv = malloc((size_t)cs->k * n * sizeof(int));
  int info = zfactor(n, B, cs, lu, piv);
  if (!info) zapply_lu(n, B, cs, form, m, R, lu, piv, out);
  free(lu); free(piv);
  return info;
}

int orc_zexpm(int n, const double complex* A, double t, const orc_coeffs* cs, int form,
              double anorm, int s_fixed, double complex* F, int* s_out) {
  size_t nn = (size_t)n * n;
  if (!all_finite(2 * nn, (const double*)A) || !isfinite(t)) return -2;
  double complex* B = malloc(nn * sizeof(double complex));
  double complex* T = malloc(nn * sizeof(double complex));
  for (size_t e = 0; e < nn; ++e) B[e] = t * A[e];
  double eta = anorm > 0.0 ? anorm * fabs(t) : orc_znorm1(n, B);
  int s = s_fixed >= 0 ? s_fixed : orc_select_s(eta, cs->theta);
  for (size_t e = 0; e < nn; ++e) B[e] = ldexp(creal(B[e]), -s) + I * ldexp(cimag(B[e]), -s);
  int info = zapply(n, B, cs, form, n, NULL, F);
  for (int q = 0; q < s && !info; ++q) {
    zmatmul(n, n, n, F, F, T);
    memcpy(F, T, nn * sizeof(double complex));
  }
  if (s_out) *s_out = s;
  free(B); free(T);
  return info;
}

int orc_zexpmv(int n, const double complex* A, double t, const orc_coeffs* cs, int form,
               double anorm, long nsteps, int m, const double complex* V, double complex* W,
               long* n_out) {
  size_t nn = (size_t)n * n, nm = (size_t)n * m;
  if (!all_finite(2 * nn, (const double*)A) || !all_finite(2 * nm, (const double*)V) ||
      !isfinite(t))
    return -2;
  double complex* B = malloc(nn * sizeof(double complex));
  double complex* Wn = malloc(nm * sizeof(double complex));
  for (size_t e = 0; e < nn; ++e) B[e] = t * A[e];
  double eta = anorm > 0.0 ? anorm * fabs(t) : orc_znorm1(n, B);
  long N = nsteps > 0 ? nsteps : orc_select_nsteps(eta, cs->theta);
  double h = t / (double)N;
  for (size_t e = 0; e < nn; ++e) B[e] = h * A[e];
  memcpy(W, V, nm * sizeof(double complex));
  /* every M_i is factored once and its factors serve all N steps (Sec. 5.1
   * remarks: the LU decomposition is done only once) */
  double complex* lu = malloc((size_t)cs->k * nn * sizeof(double complex));
  int* piv = malloc((size_t)cs->k * n * sizeof(int));
  int info = zfactor(n, B, cs, lu, piv);
  for (long q = 0; q < N && !info; ++q) {
    zapply_lu(n, B, cs, form, m, W, lu, piv, Wn);
    memcpy(W, Wn, nm * sizeof(double complex));
  }
  if (n_out) *n_out = N;
  free(B); free(Wn); free(lu); free(piv);
  return info;
}

/* ------------------------------------------------------------------------ */
/* batched drivers: independent matrices, one after another (OpenMP over    */
/* the batch when compiled with -fopenmp)                                    */
/* ------------------------------------------------------------------------ */

/* A and F packed back to back (matrix b has d[b]^2 entries at off[b]). */
int orc_expm_batched(int batch, const int* d, const long* off, const double* A,
                     const double* t, const orc_coeffs* cs, int form, double* F, int* s_out,
                     int* info) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int b = 0; b < batch; ++b) {
    info[b] = orc_expm(d[b], A + off[b], t[b], cs, form, 0.0, -1, F + off[b], s_out + b);
    bad |= (info[b] != 0);
  }
  return bad;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
