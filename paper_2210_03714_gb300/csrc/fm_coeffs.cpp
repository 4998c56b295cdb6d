// fm_coeffs.cpp -- built-in coefficient sets and the forward-bound theta.
//
// Printed sets are stored as the exact rationals of the paper (S. Blanes,
// arXiv:2210.03714) and rounded once to double.  The two phi_1 sets the paper
// does not print (R8 nodes, and R4 nodes with alpha = 5) are the exact solution
// of Eq. (LinearEqsbi), sum_i b_i c_i^k = 1/(k+1)!, k = 0..P-1, obtained here by
// Lagrange interpolation in 128-bit rational arithmetic.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <complex>

#include "../../include/fm.h"

namespace {

typedef __int128 i128;

i128 iabs128(i128 a) { return a < 0 ? -a : a; }
i128 gcd128(i128 a, i128 b) {
  a = iabs128(a);
  b = iabs128(b);
  while (b) { i128 t = a % b; a = b; b = t; }
  return a;
}

struct Q {
  i128 n, d;  // d > 0, gcd(n, d) = 1
};
Q qmk(i128 n, i128 d) {
  if (d < 0) { n = -n; d = -d; }
  i128 g = gcd128(n, d);
  if (g > 1) { n /= g; d /= g; }
  if (n == 0) d = 1;
  return {n, d};
}
Q qadd(Q a, Q b) {
  i128 g = gcd128(a.d, b.d);
  return qmk(a.n * (b.d / g) + b.n * (a.d / g), a.d / g * b.d);
}
Q qneg(Q a) { return {-a.n, a.d}; }
Q qsub(Q a, Q b) { return qadd(a, qneg(b)); }
Q qmul(Q a, Q b) {
  i128 g1 = gcd128(a.n, b.d), g2 = gcd128(b.n, a.d);
  if (g1 == 0) g1 = 1;
  if (g2 == 0) g2 = 1;
  return qmk((a.n / g1) * (b.n / g2), (a.d / g2) * (b.d / g1));
}
Q qdiv(Q a, Q b) { return qmul(a, qmk(b.d, b.n)); }

int bitlen(i128 a) {
  int l = 0;
  while (a) { ++l; a >>= 1; }
  return l;
}

// correctly rounded (to nearest, ties to even) double of n/d
double qdouble(Q q) {
  if (q.n == 0) return 0.0;
  const int neg = q.n < 0;
  const i128 a = iabs128(q.n), d = q.d;
  // quotient scaled by 2^sh so that it has 55 or 56 bits
  const int sh = 55 - (bitlen(a) - bitlen(d));
  i128 qv, r;
  if (sh >= 0) {
    qv = a / d;
    r = a % d;
    for (int i = 0; i < sh; ++i) {  // long division: r < d throughout
      r <<= 1;
      qv <<= 1;
      if (r >= d) { r -= d; qv |= 1; }
    }
  } else {
    const i128 dd = d << (-sh);
    qv = a / dd;
    r = a % dd;
  }
  const int drop = bitlen(qv) - 53;  // 2 or 3
  const i128 rem = qv & (((i128)1 << drop) - 1), half = (i128)1 << (drop - 1);
  i128 m = qv >> drop;
  if (rem > half || (rem == half && (r != 0 || (m & 1)))) m += 1;
  const double out = ldexp((double)(unsigned long long)m, drop - sh);
  return neg ? -out : out;
}

Q parse_q(const char* s) {
  i128 n = 0, d = 1;
  int neg = 0;
  if (*s == '-') { neg = 1; ++s; }
  while (*s >= '0' && *s <= '9') n = n * 10 + (*s++ - '0');
  if (*s == '/') {
    ++s;
    d = 0;
    while (*s >= '0' && *s <= '9') d = d * 10 + (*s++ - '0');
  }
  return qmk(neg ? -n : n, d);
}

Q factorial_inv(int k) {
  i128 f = 1;
  for (int i = 2; i <= k; ++i) f *= i;
  return qmk(1, f);
}

// b_i = sum_k l_{ik} a_k with l_i(x) = prod_{j != i} (x - c_j)/(c_i - c_j)
void lagrange_b(int P, const Q* c, const Q* a, Q* b) {
  for (int i = 0; i < P; ++i) {
    Q poly[32];
    poly[0] = qmk(1, 1);
    int deg = 0;
    Q den = qmk(1, 1);
    for (int j = 0; j < P; ++j) {
      if (j == i) continue;
      // poly *= (x - c_j)
      Q np[32];
      for (int t = 0; t <= deg + 1; ++t) np[t] = qmk(0, 1);
      for (int t = 0; t <= deg; ++t) {
        np[t + 1] = qadd(np[t + 1], poly[t]);
        np[t] = qsub(np[t], qmul(poly[t], c[j]));
      }
      ++deg;
      for (int t = 0; t <= deg; ++t) poly[t] = np[t];
      den = qmul(den, qsub(c[i], c[j]));
    }
    Q s = qmk(0, 1);
    for (int k = 0; k < P; ++k) s = qadd(s, qmul(poly[k], a[k]));
    b[i] = qdiv(s, den);
  }
}

struct Builtin {
  int k;
  double c_re[FM_MAX_TERMS], c_im[FM_MAX_TERMS], b_re[FM_MAX_TERMS], b_im[FM_MAX_TERMS];
  int conj_pair;
  double a0, d1, d2;
  int order;
  int func;  // 0 exp, 1 phi1
  double theta;
  int ready;
};

Builtin g_sets[FM_NUM_BUILTIN];

void set_real(Builtin& B, int k, const char* const* c, const char* const* b, const char* const* d,
              int order, int func) {
  Q cq[FM_MAX_TERMS], bq[FM_MAX_TERMS];
  Q a0 = qmk(0, 1);
  for (int i = 0; i < k; ++i) {
    cq[i] = parse_q(c[i]);
    bq[i] = parse_q(b[i]);
    a0 = qadd(a0, bq[i]);
  }
  Q dq[3] = {qmk(0, 1), qmk(0, 1), qmk(0, 1)};
  if (d)
    for (int j = 0; j < 3; ++j) dq[j] = parse_q(d[j]);
  a0 = qadd(a0, dq[0]);
  B.k = k;
  for (int i = 0; i < k; ++i) {
    B.c_re[i] = qdouble(cq[i]);
    B.c_im[i] = 0.0;
    B.b_re[i] = qdouble(bq[i]);
    B.b_im[i] = 0.0;
  }
  B.conj_pair = 0;
  B.a0 = qdouble(a0);
  B.d1 = qdouble(dq[1]);
  B.d2 = qdouble(dq[2]);
  B.order = order;
  B.func = func;
}

// exact Taylor coefficient a_k of function func (FM_FUNC_*)
Q taylor_q(int func, int k) {
  switch (func) {
    case FM_FUNC_PHI1: return factorial_inv(k + 1);
    case FM_FUNC_PHI2: return factorial_inv(k + 2);
    case FM_FUNC_COS: return k % 2 ? qmk(0, 1) : (((k / 2) % 2) ? qneg(factorial_inv(k)) : factorial_inv(k));
    case FM_FUNC_SIN: return k % 2 ? ((((k - 1) / 2) % 2) ? qneg(factorial_inv(k)) : factorial_inv(k)) : qmk(0, 1);
    case FM_FUNC_LOG1M: return k == 0 ? qmk(0, 1) : qmk(-1, k);
    default: return factorial_inv(k);
  }
}

// weights of function func on the given nodes: Eq. (LinearEqsbi) solved
// exactly (Lagrange interpolation in 128-bit rationals)
void set_derived(Builtin& B, int k, const char* const* c, int order, int func) {
  Q cq[FM_MAX_TERMS], aq[FM_MAX_TERMS], bq[FM_MAX_TERMS];
  for (int i = 0; i < k; ++i) {
    cq[i] = parse_q(c[i]);
    aq[i] = taylor_q(func, i);
  }
  lagrange_b(k, cq, aq, bq);
  Q a0 = qmk(0, 1);
  B.k = k;
  for (int i = 0; i < k; ++i) {
    B.c_re[i] = qdouble(cq[i]);
    B.c_im[i] = 0.0;
    B.b_re[i] = qdouble(bq[i]);
    B.b_im[i] = 0.0;
    a0 = qadd(a0, bq[i]);
  }
  B.conj_pair = 0;
  B.a0 = qdouble(a0);
  B.d1 = B.d2 = 0.0;
  B.order = order;
  B.func = func;
}

void set_derived_phi1(Builtin& B, int k, const char* const* c, int order) {
  Q cq[FM_MAX_TERMS], aq[FM_MAX_TERMS], bq[FM_MAX_TERMS];
  for (int i = 0; i < k; ++i) {
    cq[i] = parse_q(c[i]);
    aq[i] = factorial_inv(i + 1);  // a_k = 1/(k+1)! for phi_1
  }
  lagrange_b(k, cq, aq, bq);
  Q a0 = qmk(0, 1);
  B.k = k;
  for (int i = 0; i < k; ++i) {
    B.c_re[i] = qdouble(cq[i]);
    B.c_im[i] = 0.0;
    B.b_re[i] = qdouble(bq[i]);
    B.b_im[i] = 0.0;
    a0 = qadd(a0, bq[i]);
  }
  B.conj_pair = 0;
  B.a0 = qdouble(a0);
  B.d1 = B.d2 = 0.0;
  B.order = order;
  B.func = 1;
}

// Taylor coefficient a_k of the target function (FM_FUNC_*)
long double taylor_a(int func, int k) {
  if (func == FM_FUNC_LOG1M) return k == 0 ? 0.0L : -1.0L / (long double)k;
  if ((func == FM_FUNC_COS && k % 2) || (func == FM_FUNC_SIN && k % 2 == 0)) return 0.0L;
  long double f = 1.0L;
  int top = func == FM_FUNC_PHI1 ? k + 1 : (func == FM_FUNC_PHI2 ? k + 2 : k);
  for (int i = 2; i <= top; ++i) f *= (long double)i;
  long double v = 1.0L / f;
  if (func == FM_FUNC_COS && (k / 2) % 2) v = -v;
  if (func == FM_FUNC_SIN && ((k - 1) / 2) % 2) v = -v;
  return v;
}

void init_sets() {
  static int done = 0;
  if (done) return;
  // Sec. 4.1, Eq. (Frac4ci) with alpha = 5 and Eq. (Frac4bi)
  static const char* r4c[] = {"0", "1/5", "-1/5", "1/10", "-1/10"};
  static const char* r4b[] = {"128/3", "85/3", "20/9", "-515/9", "-15"};
  set_real(g_sets[FM_R4], 5, r4c, r4b, nullptr, 4, 0);
  // Sec. 4.1, phi_1 with alpha = 6
  static const char* r4pc[] = {"0", "1/6", "-1/6", "1/12", "-1/12"};
  static const char* r4pb[] = {"71/5", "117/10", "7/10", "-104/5", "-24/5"};
  set_real(g_sets[FM_R4_PHI1], 5, r4pc, r4pb, nullptr, 4, 1);
  set_derived_phi1(g_sets[FM_R4_PHI1_A5], 5, r4c, 4);
  // Sec. 4.2, Eq. (Frac8ci) with alpha = 5 and Eq. (Frac8bi)
  static const char* r8c[] = {"0", "1/5", "-1/5", "2/15", "-2/15", "1/10", "-1/10", "2/25", "-2/25"};
  static const char* r8b[] = {"-9979069/32256",   "-1995521/254016",        "-392009/254016",
                              "520866369/802816", "48898161/802816",        "-26686735/11907",
                              "-3892615/11907",   "353067578125/195084288", "71873828125/195084288"};
  set_real(g_sets[FM_R8], 9, r8c, r8b, nullptr, 8, 0);
  set_derived_phi1(g_sets[FM_R8_PHI1], 9, r8c, 8);
  // Sec. 1: cos, sin (double-angle formulae) and phi_2 on the R8 nodes
  set_derived(g_sets[FM_R8_COS], 9, r8c, 8, FM_FUNC_COS);
  set_derived(g_sets[FM_R8_SIN], 9, r8c, 8, FM_FUNC_SIN);
  set_derived(g_sets[FM_R8_PHI2], 9, r8c, 8, FM_FUNC_PHI2);
  // Sec. 2, Eq. (Frac4bi0) and the two sets printed after it: c_i = 1/(i+1)
  static const char* f4c[] = {"1/2", "1/3", "1/4", "1/5", "1/6"};
  static const char* f4e[] = {"1/3", "-18", "128", "-625/3", "99"};
  static const char* f4p[] = {"7/18", "-9", "128/3", "-500/9", "45/2"};
  static const char* f4l[] = {"-35/3", "153/2", "-160", "625/6", "-9"};
  set_real(g_sets[FM_FRAC4_EXP], 5, f4c, f4e, nullptr, 4, FM_FUNC_EXP);
  set_real(g_sets[FM_FRAC4_PHI1], 5, f4c, f4p, nullptr, 4, FM_FUNC_PHI1);
  set_real(g_sets[FM_FRAC4_LOG1M], 5, f4c, f4l, nullptr, 4, FM_FUNC_LOG1M);
  // Sec. 5.1, Eq. (Frac5bi0)
  static const char* r5c[] = {"0", "1/3", "1/4", "1/5", "1/6", "1/7"};
  static const char* r5b[] = {"-43/12", "81/32", "-704/9", "23125/48", "-810", "117649/288"};
  set_real(g_sets[FM_R5], 6, r5c, r5b, nullptr, 5, 0);
  // Sec. 4.3.1, Eq. (Frac10ci)/(Frac10bi); the printed "d_1, d_2, d_3" are the
  // d_0, d_1, d_2 of Eq. (Frac10)
  static const char* r10c[] = {"-1/8", "1/8", "-1/10", "1/10", "-1/12", "1/12", "-1/14", "1/14", "-1/16", "1/16"};
  static const char* r10b[] = {"-57383239/760320",          "-115498838729/239500800",
                               "1648441938671875/1255673954304", "56790060546875/4227858432",
                               "-1476772203681/298188800",  "-31012455666807/656015360",
                               "4891212112962371/1295536619520", "171190903245297593/3886609858560",
                               "2000", "-3500"};
  static const char* r10d[] = {"-781562376863/94371840", "-54849495983/330301440", "-8034429391/587202560"};
  set_real(g_sets[FM_R10], 10, r10c, r10b, r10d, 10, 0);
  // Sec. 4.3.1, Eq. (Frac10ciNO)/(Frac10biNO)
  static const char* r10sc[] = {"1/7", "1/8", "1/9", "1/10", "1/11", "1/12", "1/13", "1/14", "1/15", "1/16"};
  static const char* r10sb[] = {"-2385751622325187262153/1585084524134400000",
                                "3752603696192081/82668600000",
                                "-87230538798639033213/187904819200000",
                                "14789110319838821875/6934744793088",
                                "-10558563753676365149296981/2219118333788160000",
                                "3520134037769971/716800000",
                                "-2263057299714115181019509/1585084524134400000",
                                "-2275831141003773874927/3095868211200000",
                                "-50000", "350000"};
  static const char* r10sd[] = {"-34244933704346617/14676708556800", "-18541933026870559/428070666240000",
                                "-6798371473106351/15410543984640000"};
  set_real(g_sets[FM_R10_STAR], 10, r10sc, r10sb, r10sd, 10, 0);
  // Eq. (Pade4): 1 + 2 Re(w/(x - z)), z = 3 - i sqrt(3), w = 6 + 6 sqrt(3) i
  // (the residue is printed as 6 sqrt(6); 6 sqrt(3) is the value that equals
  // the left-hand side of the same equation).  As b/(1 - c x): c = 1/z, b = -w/z.
  {
    Builtin& B = g_sets[FM_PADE22];
    std::complex<long double> z(3.0L, -sqrtl(3.0L)), w(6.0L, 6.0L * sqrtl(3.0L));
    std::complex<long double> c = 1.0L / z, b = -w / z;
    B.k = 1;
    B.c_re[0] = (double)c.real();
    B.c_im[0] = (double)c.imag();
    B.b_re[0] = 0.0;  // -w/z = -2 sqrt(3) i exactly
    B.b_im[0] = (double)b.imag();
    B.conj_pair = 1;
    B.a0 = 1.0;  // 1 + 2 Re(b)
    B.d1 = B.d2 = 0.0;
    B.order = 4;
    B.func = 0;
  }
  // Eq. (Pade4phi1): 1/3 + 2 Re((7/3 + 8i)/(x - (4 - 2i))): c = 0.2 + 0.1i,
  // b = 1/3 - 11/6 i
  {
    Builtin& B = g_sets[FM_PADE22_PHI1];
    B.k = 1;
    B.c_re[0] = 0.2;
    B.c_im[0] = 0.1;
    B.b_re[0] = 1.0 / 3.0;
    B.b_im[0] = -11.0 / 6.0;
    B.conj_pair = 1;
    B.a0 = 1.0;  // 1/3 + 2/3
    B.d1 = B.d2 = 0.0;
    B.order = 4;
    B.func = 1;
  }
  for (int id = 0; id < FM_NUM_BUILTIN; ++id) {
    fm_coeffs cs;
    Builtin& B = g_sets[id];
    cs.k = B.k;
    cs.c_re = B.c_re;
    cs.c_im = B.c_im;
    cs.b_re = B.b_re;
    cs.b_im = B.b_im;
    cs.conj_pair = B.conj_pair;
    cs.a0 = B.a0;
    cs.d1 = B.d1;
    cs.d2 = B.d2;
    cs.order = B.order;
    cs.theta = 0;
    double th = 0;
    fm_theta(&cs, B.func, ldexp(1.0, -53), &th);
    B.theta = th;
    B.ready = 1;
  }
  done = 1;
}

}  // namespace

extern "C" fm_status fm_theta(const fm_coeffs* cs, int func, double tol, double* theta_out) {
  if (!cs || !theta_out || cs->k < 1 || cs->k > FM_MAX_TERMS || !(tol > 0) || func < 0 ||
      func > FM_FUNC_LOG1M)
    return FM_EINVAL;
  // alpha_k = sum_i b_i c_i^k (+ d_k for k <= 2, d0 = a0 - sum b_i), Sec. 3
  const int K = 200;
  static long double gam[200];
  long double sb = 0;
  for (int i = 0; i < cs->k; ++i) sb += cs->conj_pair ? 2.0L * cs->b_re[i] : cs->b_re[i];
  for (int k = 0; k < K; ++k) {
    long double al = 0;
    for (int i = 0; i < cs->k; ++i) {
      std::complex<long double> c(cs->c_re[i], cs->c_im ? cs->c_im[i] : 0.0);
      std::complex<long double> b(cs->b_re[i], cs->b_im ? cs->b_im[i] : 0.0);
      std::complex<long double> p = b * std::pow(c, k);
      al += cs->conj_pair ? 2.0L * p.real() : p.real();
    }
    if (k == 0) al += (long double)cs->a0 - sb;
    if (k == 1) al += cs->d1;
    if (k == 2) al += cs->d2;
    gam[k] = k > cs->order ? fabsl(taylor_a(func, k) - al) : 0.0L;
  }
  auto eps = [&](long double x) {
    long double s = 0, p = 1;
    for (int k = 0; k < K; ++k) {
      s += gam[k] * p;
      p *= x;
    }
    return s;
  };
  long double lo = 0, hi = 1;
  while (eps(hi) < tol && hi < 1e6) hi *= 2;
  for (int it = 0; it < 200; ++it) {
    long double mid = 0.5L * (lo + hi);
    if (eps(mid) < tol) lo = mid; else hi = mid;
  }
  *theta_out = (double)lo;
  return FM_OK;
}

extern "C" fm_status fm_coeffs_builtin(int id, fm_coeffs* out) {
  if (id < 0 || id >= FM_NUM_BUILTIN || !out) return FM_EINVAL;
  init_sets();
  Builtin& B = g_sets[id];
  out->k = B.k;
  out->c_re = B.c_re;
  out->c_im = B.c_im;
  out->b_re = B.b_re;
  out->b_im = B.b_im;
  out->conj_pair = B.conj_pair;
  out->a0 = B.a0;
  out->d1 = B.d1;
  out->d2 = B.d2;
  out->order = B.order;
  out->theta = B.theta;
  return FM_OK;
}
