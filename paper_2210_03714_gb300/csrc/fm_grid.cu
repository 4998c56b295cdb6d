// fm_grid.cu -- the grid-wide path: one matrix of large order spread over
// every SM, as a stream-ordered sequence of kernels (grid.cuh).
//
// For each shift c_i the system (I - C) Y = C, C = c_i B, is solved by the
// residual-correction iteration
//     E = C - (I - C) Y        (residual of the current Y)
//     Y <- Y + (I + Y) E        (correction through the current inverse I + Y)
// starting from Y = C: Newton-Schulz for (I - C)^{-1} = I + Y, written in the
// deviation Y so both products act on small matrices.  Y converges to
// (I - C)^{-1} C, the term of the roundoff form (Eq. ParallRoundOff), with the
// residual squaring each time (||E|| ~ ||C||^(2^(j+1))); the paper's sets
// keep ||c_i B||_1 <= 0.05, so three iterations reach double precision.
// Then F = a0 I + d1 B + d2 B^2 + sum_i b_i Y_i (Sec. 2) and, in the
// deviation E = F - I: s squarings E <- 2E + E E (Sec. 1), phi_1 doublings,
// or N steps W <- W + E W for the action (Sec. 1; the matrix r(B) is formed
// once and reused by every step).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "../../include/fm.h"
#include "fm_grid.h"
#include "grid.cuh"

namespace fmk {
namespace {

constexpr int kThreads = 256;

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }
int rnd(int x, int q) { return (x + q - 1) / q * q; }

struct Layout {
  size_t B, C, Y, E, F0, F1, B2, B4, B6, G, Tm, colsum, misc, rmax, cmax, ex, fy, px, py, acc, total;
  size_t pxs, pys;
};

Layout layout(int kind, bool cplx, int precision, int d, int m) {
  Layout L;
  memset(&L, 0, sizeof L);
  const size_t elt = cplx ? 16 : 8;
  const bool act = kind == JOB_EXPMV || kind == JOB_PHI1MV;
  const int w = act && m > d ? m : d;
  const size_t nn = (size_t)d * d * elt;
  const int Mp = rnd(d, oz::TM), Np = rnd(w, oz::TN);
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o += up(b);
    return at;
  };
  L.B = take(nn);
  L.C = take(nn);
  L.Y = take(nn);
  L.E = take(nn);
  L.F0 = take(nn);
  const bool two = kind == JOB_PHI1 || kind == JOB_PHI1MV || kind == JOB_TRIG;
  L.F1 = take(two ? nn : 0);
  L.B2 = take(nn);
  L.B4 = take(nn);
  L.B6 = take(nn);
  L.G = take((two ? 2 : 1) * nn);
  L.Tm = take(precision == 0 ? (size_t)d * w * elt : 0);
  L.colsum = take((size_t)d * 8);
  L.misc = take(256);
  L.rmax = take((size_t)Mp * 8);
  L.cmax = take((size_t)Np * 8);
  L.ex = take((size_t)Mp * 4);
  L.fy = take((size_t)Np * 4);
  if (precision != 0) {
    const int kc = (d + grid::GKC - 1) / grid::GKC;
    L.pxs = (size_t)(Mp / oz::TM) * kc * grid::GXST;
    L.pys = (size_t)(Np / oz::TN) * kc * grid::GYST;
    L.px = take(L.pxs * (cplx ? 2 : 1));
    L.py = take(L.pys * (cplx ? 3 : 1));
    L.acc = take((size_t)(cplx ? 2 : 1) * Mp * Np * 16);
  }
  L.total = o;
  return L;
}

int sms_of_device() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// misc words on the device
struct Misc {
  int nonfinite;
  int tc_err;
  int pad[2];
  double eta;
  unsigned long long emax;
  unsigned long long emax4;  // largest entry of B^4 (bits)
};

template <class T>
class Runner {
 public:
  Runner(const GridJob& g, char* msg, size_t len) : g_(g), msg_(msg), len_(len) {}

  int run();

 private:
  const GridJob& g_;
  char* msg_;
  size_t len_;
  cudaStream_t st_ = nullptr;
  int n_ = 0, sms_ = 1;
  bool tcp_ = false;
  Layout L_;
  char* base_ = nullptr;
  T *B_ = nullptr, *C_ = nullptr, *Y_ = nullptr, *E_ = nullptr, *F0_ = nullptr, *F1_ = nullptr,
    *B2_ = nullptr, *B4_ = nullptr, *B6_ = nullptr, *G_ = nullptr, *Tm_ = nullptr;
  double* colsum_ = nullptr;
  Misc* misc_ = nullptr;
  unsigned long long *rmax_ = nullptr, *cmax_ = nullptr;
  int *ex_ = nullptr, *fy_ = nullptr;
  unsigned char *px_ = nullptr, *py_ = nullptr;
  long long* acc_ = nullptr;
  cudaError_t err_ = cudaSuccess;
  fm_stats* stats_ = nullptr;
  TileTimer timer_;

  int blocks(size_t count) const {
    size_t b = (count + kThreads - 1) / kThreads;
    size_t cap = (size_t)sms_ * 8;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
  }
  long long launches_ = 0;
  void check(const char* where) {
    ++launches_;
    if (err_ != cudaSuccess) return;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      err_ = e;
      snprintf(msg_, len_, "%s: %s", where, cudaGetErrorString(e));
    }
  }
  void memset0(void* p, size_t bytes, const char* where) {
    if (err_ != cudaSuccess) return;
    cudaError_t e = cudaMemsetAsync(p, 0, bytes, st_);
    if (e != cudaSuccess) {
      err_ = e;
      snprintf(msg_, len_, "%s: %s", where, cudaGetErrorString(e));
    }
  }
  Misc read_misc() {
    Misc h;
    memset(&h, 0, sizeof h);
    if (err_ != cudaSuccess) return h;
    cudaError_t e = cudaMemcpyAsync(&h, misc_, sizeof h, cudaMemcpyDeviceToHost, st_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
    if (e != cudaSuccess) {
      err_ = e;
      snprintf(msg_, len_, "reading the status: %s", cudaGetErrorString(e));
    }
    return h;
  }

  // out (M x N, ldo) = epilogue(X (M x K) Y (K x N)); split_x = false reuses
  // the row digit planes of the previous product's X (same matrix, same M, K)
  void prod(int M, int N, int K, const T* X, int ldx, bool split_x, const T* Yp, int ldy,
            const grid::Epi& e_in, T* out, int ldo, int lmax = 8) {
    if (err_ != cudaSuccess) return;
    grid::Epi e = e_in;
    grid::fixed_form(e);
    if (stats_) {
      const double f = (grid::El<T>::parts == 2 ? 8.0 : 2.0) * M * (double)N * K;
      stats_->products += 1;
      stats_->product_flops += f;
      if (tcp_) stats_->digit_flops += f * (lmax - 1) * lmax / 2;  // digit pairs kept
    }
    if (!tcp_) {
      const int tiles = ((M + GT - 1) / GT) * ((N + GT - 1) / GT);
      grid::dgemm_tiles<T><<<tiles, NT, 0, st_>>>(M, N, K, X, ldx, Yp, ldy, Tm_, N);
      check("FP64 product");
      grid::epilogue<T><<<blocks((size_t)M * N), kThreads, 0, st_>>>(
          M, N, nullptr, 1, 0, 0, nullptr, nullptr, Tm_, N, e, out, ldo);
      check("product epilogue");
      return;
    }
    const int parts = grid::El<T>::parts;
    const int kc = (K + grid::GKC - 1) / grid::GKC;
    const int mtn = (M + oz::TM - 1) / oz::TM, ntn = (N + oz::TN - 1) / oz::TN;
    const int Mp = mtn * oz::TM, Np = ntn * oz::TN;
    // plane-set strides for this K (the buffers are sized for K = d)
    const size_t pxs = (size_t)mtn * kc * grid::GXST, pys = (size_t)ntn * kc * grid::GYST;
    if (split_x) {
      memset0(rmax_, (size_t)M * 8, "row maxima reset");
      grid::row_max<T><<<blocks((size_t)M * 32), kThreads, 0, st_>>>(M, K, X, ldx, rmax_);
      check("row maxima");
      const size_t items = (size_t)Mp * kc * (grid::GKC / 8);
      grid::split_rows<T><<<blocks(items), kThreads, 0, st_>>>(M, K, X, ldx, rmax_, px_, pxs, kc, ex_);
      check("row digit planes");
    }
    memset0(cmax_, (size_t)N * 8, "column maxima reset");
    {
      dim3 gdim((N + 31) / 32, 1);
      int gy = (sms_ * 4 + (int)gdim.x - 1) / (int)gdim.x;
      int gymax = (K + 7) / 8;
      gdim.y = gy < 1 ? 1 : (gy > gymax ? gymax : gy);
      grid::col_max<T><<<gdim, kThreads, 0, st_>>>(K, N, Yp, ldy, cmax_);
      check("column maxima");
    }
    {
      const size_t items = (size_t)Np * kc * (grid::GKC / 8);
      grid::split_cols<T><<<blocks(items), kThreads, 0, st_>>>(K, N, Yp, ldy, cmax_, py_, pys, kc, fy_);
      check("column digit planes");
    }
    grid::OzTiles a;
    memset(&a, 0, sizeof a);
    a.px = px_;
    a.py = py_;
    a.pxs = pxs;
    a.pys = pys;
    a.mtn = mtn;
    a.ntn = ntn;
    a.kc = kc;
    a.nparts = parts;
    a.nseg = parts;
    if (parts == 1) {
      a.sx[0][0] = 0;
      a.sy[0][0] = 0;
    } else {
      // re = Xr Yr + Xi (-Yi);  im = Xr Yi + Xi Yr
      a.sx[0][0] = 0; a.sy[0][0] = 0;
      a.sx[0][1] = 1; a.sy[0][1] = 2;
      a.sx[1][0] = 0; a.sy[1][0] = 1;
      a.sx[1][1] = 1; a.sy[1][1] = 0;
    }
    const int tiles = parts * mtn * ntn;
    const int groups = (a.nseg * kc + grid::GSTEPS - 1) / grid::GSTEPS;
    // split K so the CTAs fill whole waves: estimated time = waves x (groups
    // per CTA + about 1.5 groups of fixed cost per CTA)
    int ksplit = 1;
    double best = 1e300;
    for (int ks = 1; ks <= groups && ks <= 32; ++ks) {
      const long long ctas = (long long)tiles * ks;
      const double waves = (double)((ctas + sms_ - 1) / sms_);
      const double est = waves * ((double)((groups + ks - 1) / ks) + 1.5);
      if (est < best - 1e-9) {
        best = est;
        ksplit = ks;
      }
    }
    a.ksplit = ksplit;
    a.lmax = lmax;
    a.acc = acc_;
    a.err = &misc_->tc_err;
    memset0(acc_, (size_t)parts * Mp * Np * 16, "accumulator reset");
    a.nitems = tiles * ksplit;
    const int ctas = a.nitems < sms_ ? a.nitems : sms_;  // persistent: one CTA per SM
    timer_.start(st_);
    grid::oz_tiles<<<ctas, grid::GTHREADS, grid::GSMEM + 1024, st_>>>(a);
    timer_.stop(st_);
    check("tensor-core product");
    grid::epilogue<T><<<blocks((size_t)M * N), kThreads, 0, st_>>>(
        M, N, acc_, parts, Mp, Np, ex_, fy_, nullptr, 0, e, out, ldo);
    check("product epilogue");
  }

  // E <- 2E + E E  (one squaring of F = I + E)
  void square(T* E) {
    grid::Epi e;
    e.Z1 = E;
    e.ld1 = n_;
    e.b1r = 2.0;
    prod(n_, n_, n_, E, n_, true, E, n_, e, E, n_);
  }
};

template <class T>
int Runner<T>::run() {
  const GridJob& g = g_;
  st_ = g.st;
  n_ = g.d;
  stats_ = (fm_stats*)g.stats;
  if (stats_) memset(stats_, 0, sizeof *stats_);
  sms_ = sms_of_device();
  tcp_ = g.precision != 0;
  const int n = n_;
  const bool act = g.kind == JOB_EXPMV || g.kind == JOB_PHI1MV;
  const bool phi = g.kind == JOB_PHI1 || g.kind == JOB_PHI1MV;
  const bool trig = g.kind == JOB_TRIG;  // cos in F0, sin in F1
  const bool two = phi || trig;
  L_ = layout(g.kind, g.cplx, g.precision, n, g.m);
  if (g.ws_bytes < L_.total) {
    snprintf(msg_, len_, "grid path: workspace too small");
    return FM_ENOMEM;
  }
  base_ = (char*)g.ws;
  B_ = (T*)(base_ + L_.B);
  C_ = (T*)(base_ + L_.C);
  Y_ = (T*)(base_ + L_.Y);
  E_ = (T*)(base_ + L_.E);
  F0_ = (T*)(base_ + L_.F0);
  F1_ = two ? (T*)(base_ + L_.F1) : nullptr;
  B2_ = (T*)(base_ + L_.B2);
  B4_ = (T*)(base_ + L_.B4);
  B6_ = (T*)(base_ + L_.B6);
  G_ = (T*)(base_ + L_.G);
  Tm_ = tcp_ ? nullptr : (T*)(base_ + L_.Tm);
  colsum_ = (double*)(base_ + L_.colsum);
  misc_ = (Misc*)(base_ + L_.misc);
  rmax_ = (unsigned long long*)(base_ + L_.rmax);
  cmax_ = (unsigned long long*)(base_ + L_.cmax);
  ex_ = (int*)(base_ + L_.ex);
  fy_ = (int*)(base_ + L_.fy);
  if (tcp_) {
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
      cudaError_t e = cudaFuncSetAttribute(grid::oz_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           grid::GSMEM + 1024);
      if (e != cudaSuccess) {
        snprintf(msg_, len_, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        return FM_ECUDA;
      }
      attr_set[dev] = true;
    }
    px_ = (unsigned char*)(base_ + L_.px);
    py_ = (unsigned char*)(base_ + L_.py);
    acc_ = (long long*)(base_ + L_.acc);
  }
  const size_t nn = (size_t)n * n;
  const T* A = (const T*)g.A;
  const FmCoef& cf = g.cf;

  // a1: B = tA, eta = ||tA||_1, finiteness of A (and V)
  memset0(misc_, sizeof(Misc), "status reset");
  grid::colsum_scale<T><<<(n + 127) / 128, 128, 0, st_>>>(n, A, g.lda, g.t, B_, colsum_,
                                                          &misc_->nonfinite);
  check("norm");
  grid::colsum_max<<<1, 1024, 0, st_>>>(n, colsum_, &misc_->eta);
  check("norm reduction");
  if (act)
    grid::copy_check<T><<<blocks((size_t)n * g.m), kThreads, 0, st_>>>(
        n, g.m, (const T*)g.V, g.ldv, (T*)g.W, g.ldw, &misc_->nonfinite);
  check("copy of V");
  Misc h = read_misc();
  if (err_ != cudaSuccess) return FM_ECUDA;
  int info = (h.nonfinite || !isfinite(g.t)) ? -2 : 0;
  const double eta = g.anorm > 0 ? g.anorm * fabs(g.t) : h.eta;
  int s = 0;
  long long N = 0;
  if (act && g.kind == JOB_EXPMV) {
    N = g.nsteps;
    if (N <= 0) {
      const double qn = ceil(eta / cf.theta);
      N = qn < 1.0 ? 1 : (long long)qn;
    }
  } else {
    if (g.s_fixed >= 0) {
      s = g.s_fixed;
    } else if (g.s_fixed == kSRfun) {
      s = 0;  // r(tA) as it is: no range reduction
      if (info == 0 && !(eta <= cf.theta)) info = -5;
    } else {
      while (eta > ldexp(cf.theta, s) && s < 1023) ++s;
    }
  }
  auto finish = [&](int inf) -> int {
    if (err_ != cudaSuccess) return FM_ECUDA;
    cudaError_t e = cudaStreamSynchronize(st_);
    if (e != cudaSuccess) {
      snprintf(msg_, len_, "grid path: %s", cudaGetErrorString(e));
      return FM_ECUDA;
    }
    if (g.info_host) *g.info_host = inf;
    if (g.s_host) *g.s_host = s;
    if (g.n_host) *g.n_host = act && g.kind == JOB_EXPMV ? (long)N : (long)s;
    return FM_OK;
  };
  if (info == -2) return finish(info);

  // a2: B = tA / 2^s, or B = (t/N) A for the action
  if (g.kind == JOB_EXPMV) {
    grid::scale_into<T><<<blocks(nn), kThreads, 0, st_>>>(n, A, g.lda, g.t / (double)N, B_);
    check("scaling");
  } else {
    grid::pow2_scale<T><<<blocks(nn), kThreads, 0, st_>>>(nn, B_, s);
    check("scaling");
  }

  // a3-a6 plan: one system per nonzero node; a pair of nodes +c, -c of the
  // roundoff form shares one system I - c^2 B^2, a term of a conjugate-pair set
  // is one real system I - 2 Re(c) B + |c|^2 B^2 (Sec. 1: one product, x^2, and
  // one inverse per pair of roots)
  const int nf = two ? 2 : 1;
  Sys sys[kMaxTerms];
  double base[2];
  const int nsys = plan_systems(cf, g.form, true, sys, base);
  bool any_quad = false;
  for (int q = 0; q < nsys; ++q) {
    any_quad |= sys[q].quad != 0;
    // a quadratic system's g I (plain form) joins the starting multiple of I
    if (sys[q].quad)
      for (int f = 0; f < nf; ++f) base[f] += sys[q].gr[f];
  }
  // a6 (first part): F_f = base_f I + d1 B + d2 B^2
  const bool need_b2 = cf.d2[0] != 0 || (two && cf.d2[1] != 0) || any_quad;
  if (need_b2) {
    grid::Epi e;
    prod(n, n, n, B_, n, true, B_, n, e, B2_, n);
  }
  for (int f = 0; f < nf; ++f) {
    grid::init_f<T><<<blocks(nn), kThreads, 0, st_>>>(n, base[f], cf.d1[f], B_, cf.d2[f],
                                                       need_b2 ? B2_ : nullptr, f ? F1_ : F0_);
    check("initial combination");
  }

  // systems C = u B^2 with u real (the fused +-c pairs) take their first
  // correction step from B^4 = B^2 B^2 and B^6 = B^4 B^2, formed once
  auto shared_ok = [](const Sys& S) {
    return S.quad && S.u1r == 0.0 && S.u1i == 0.0 && S.u2i == 0.0;
  };
  int nshared = 0;
  for (int q = 0; q < nsys; ++q) nshared += shared_ok(sys[q]) ? 1 : 0;
  double em4 = 0.0;
  if (nshared > 0) {
    memset0(&misc_->emax4, 8, "maximum reset");
    grid::Epi e4;
    e4.maxabs = &misc_->emax4;
    prod(n, n, n, B2_, n, true, B2_, n, e4, B4_, n);
    grid::Epi e6;
    prod(n, n, n, B4_, n, true, B2_, n, e6, B6_, n);
    const Misc h4 = read_misc();
    memcpy(&em4, &h4.emax4, sizeof em4);
  }

  // a3-a5: every shifted system, ascending first term; a6: F_f += b_i Y_i
  const double stop = ldexp(1.0, -30) / (double)n;
  bool pair_seen = false;
  double asum_r[2] = {0.0, 0.0}, asum_i[2] = {0.0, 0.0};
  for (int qs = 0; qs < nsys && err_ == cudaSuccess; ++qs) {
    const Sys& S = sys[qs];
    double prev = INFINITY;
    int it0 = 0;
    bool done = false;
    if (nshared > 0 && shared_ok(S)) {
      // step 0 from the shared powers: the residual u^2 B^4, its largest entry
      // u^2 max|B^4|, the same decisions as below
      const double u = S.u2r, u2 = u * u, u3 = u2 * u;
      const double em = em4 * u2;
      grid::pair_first<T><<<blocks(nn), kThreads, 0, st_>>>(nn, u, u2, u3, B2_, B4_, B6_, C_, Y_);
      check("first correction");
      if (em == 0.0) {
        done = true;
      } else if (!(em < INFINITY) || g.max_iters <= 0) {
        if (info == 0) info = -1;
        done = true;
      } else {
        prev = em;
        if (stats_ && stats_->corrections < 1) stats_->corrections = 1;
        done = em <= stop;
        it0 = 1;
      }
    } else {
      if (S.quad)  // C = u1 B + u2 B^2
        grid::build_shift2<T><<<blocks(nn), kThreads, 0, st_>>>(nn, B_, S.u1r, S.u1i, B2_, S.u2r,
                                                                S.u2i, C_, Y_);
      else
        grid::build_shift<T><<<blocks(nn), kThreads, 0, st_>>>(nn, B_, S.cr, S.ci, C_, Y_);
      check("shift");
    }
    for (int it = it0; !done; ++it) {
      // E = C Y + C - Y  (= C - (I - C) Y), and its largest entry
      memset0(&misc_->emax, 8, "residual maximum reset");
      grid::Epi e1;
      e1.Z1 = C_;
      e1.ld1 = n;
      e1.b1r = 1.0;
      e1.Z2 = Y_;
      e1.ld2 = n;
      e1.b2r = -1.0;
      e1.maxabs = &misc_->emax;
      prod(n, n, n, C_, n, true, Y_, n, e1, E_, n);  // (Y E below overwrites the row planes)
      Misc hm = read_misc();
      if (err_ != cudaSuccess) break;
      double em;
      memcpy(&em, &hm.emax, sizeof em);
      if (em == 0.0) break;
      if (!(em < INFINITY) || it >= g.max_iters || (it >= 3 && em >= prev)) {
        if (info == 0) info = -1;
        break;
      }
      prev = em;
      if (stats_ && it + 1 > stats_->corrections) stats_->corrections = it + 1;
      // Y = Y E + Y + E  (= Y + (I + Y) E).  Y E needs an absolute accuracy of
      // about u max|Y|; its error is about 2^(14 - 8 Lmax) 8 sqrt(d) max|Y| max|E|:
      // keep the digit-pair levels that bound requires
      int lmax = 8;
      if (em < 1) {
        lmax = (int)ceil((70.0 + 0.5 * log2((double)n) + log2(em)) / 8.0);
        lmax = lmax < 2 ? 2 : (lmax > 8 ? 8 : lmax);
      }
      grid::Epi e2;
      e2.Z1 = Y_;
      e2.ld1 = n;
      e2.b1r = 1.0;
      e2.Z2 = E_;
      e2.ld2 = n;
      e2.b2r = 1.0;
      prod(n, n, n, Y_, n, true, E_, n, e2, Y_, n, lmax);
      if (em <= stop) break;  // the residual after this correction is ~em^2
    }
    for (int f = 0; f < nf && err_ == cudaSuccess; ++f) {
      T* Ff = f ? F1_ : F0_;
      if (S.quad) {
        // (I + Y)(g I + a B + b B^2) = g I + y Y + x (I + Y) B with Y = M^-1 - I:
        // F += y Y now (g I is in base), G += x Y, and x B + G B after the last one
        grid::pair_acc<T><<<blocks(nn), kThreads, 0, st_>>>(nn, S.yr[f], S.yi[f], S.xr[f], S.xi[f],
                                                           Y_, !pair_seen, Ff, G_ + (size_t)f * nn);
        check("pair combination");
        asum_r[f] += S.xr[f];
        asum_i[f] += S.xi[f];
      } else {
        grid::accumulate<T><<<blocks(nn), kThreads, 0, st_>>>(n, S.wr[f], S.wi[f], Y_, g.form == 1,
                                                             Ff);
        check("combination");
      }
    }
    if (S.quad) pair_seen = true;
  }
  // the pairs' a B + G B: one product per function, F = G B + F + (sum a) B
  for (int f = 0; f < nf && pair_seen && err_ == cudaSuccess; ++f) {
    T* Ff = f ? F1_ : F0_;
    grid::Epi e;
    e.Z1 = Ff;
    e.ld1 = n;
    e.b1r = 1.0;
    e.Z2 = B_;
    e.ld2 = n;
    e.b2r = asum_r[f];
    e.b2i = asum_i[f];
    prod(n, n, n, G_ + (size_t)f * nn, n, true, B_, n, e, Ff, n);
  }
  if (err_ != cudaSuccess) return FM_ECUDA;

  // a7, in the deviation from the identity: E = F0 - I (and Psi = F1 - I)
  grid::add_identity<T><<<blocks(nn), kThreads, 0, st_>>>(n, n, F0_, n, -1.0, E_, n);
  check("deviation");
  if (phi) {
    grid::add_identity<T><<<blocks(nn), kThreads, 0, st_>>>(n, n, F1_, n, -1.0, F1_, n);
    check("deviation");
  }
  if (g.kind == JOB_EXPM) {
    for (int q = 0; q < s; ++q) square(E_);
    grid::add_identity<T><<<blocks(nn), kThreads, 0, st_>>>(n, n, E_, n, 1.0, (T*)g.F, g.ldf);
    check("output");
  } else if (trig) {
    // double angle (Sec. 1) with C = I + X: S <- 2 S C = 2S + 2 X S,
    // X <- 2 C^2 - 2I = 4X + 2 X X
    T* S = F1_;
    for (int q = 0; q < s; ++q) {
      grid::Epi e1;
      e1.ar = 2.0;
      e1.Z1 = S;
      e1.ld1 = n;
      e1.b1r = 2.0;
      prod(n, n, n, E_, n, true, S, n, e1, S, n);
      grid::Epi e2;
      e2.ar = 2.0;
      e2.Z1 = E_;
      e2.ld1 = n;
      e2.b1r = 4.0;
      prod(n, n, n, E_, n, false, E_, n, e2, E_, n);
    }
    grid::add_identity<T><<<blocks(nn), kThreads, 0, st_>>>(n, n, E_, n, 1.0, (T*)g.F, g.ldf);
    check("output");
    if (g.E) {
      grid::add_identity<T><<<blocks(nn), kThreads, 0, st_>>>(n, n, S, n, 0.0, (T*)g.E, g.lde);
      check("output");
    }
  } else if (phi) {
    // (Phi, E) <- ((E + I) Phi / 2, E^2):  Psi <- Psi + E/2 + E Psi / 2,  E <- 2E + E E
    T* Psi = F1_;
    for (int q = 0; q < s; ++q) {
      grid::Epi e1;
      e1.ar = 0.5;
      e1.Z1 = Psi;
      e1.ld1 = n;
      e1.b1r = 1.0;
      e1.Z2 = E_;
      e1.ld2 = n;
      e1.b2r = 0.5;
      prod(n, n, n, E_, n, true, Psi, n, e1, Psi, n);
      grid::Epi e2;
      e2.Z1 = E_;
      e2.ld1 = n;
      e2.b1r = 2.0;
      prod(n, n, n, E_, n, false, E_, n, e2, E_, n);
    }
    if (g.kind == JOB_PHI1) {
      grid::add_identity<T><<<blocks(nn), kThreads, 0, st_>>>(n, n, Psi, n, 1.0, (T*)g.F, g.ldf);
      check("output");
      if (g.E) {
        grid::add_identity<T><<<blocks(nn), kThreads, 0, st_>>>(n, n, E_, n, 1.0, (T*)g.E, g.lde);
        check("output");
      }
    } else {
      // W = Phi V = V + Psi V
      grid::Epi e;
      e.Z1 = g.V;
      e.ld1 = g.ldv;
      e.b1r = 1.0;
      prod(n, g.m, n, Psi, n, true, (const T*)g.V, g.ldv, e, (T*)g.W, g.ldw);
    }
  } else {
    // N steps W <- r(B) W = W + E W, the row digit planes of E split once
    for (long long q = 0; q < N && err_ == cudaSuccess; ++q) {
      grid::Epi e;
      e.Z1 = g.W;
      e.ld1 = g.ldw;
      e.b1r = 1.0;
      prod(n, g.m, n, E_, n, q == 0, (const T*)g.W, g.ldw, e, (T*)g.W, g.ldw);
    }
  }
  Misc hf = read_misc();
  if (err_ != cudaSuccess) return FM_ECUDA;
  if (hf.tc_err) info = -7;
  if (stats_) {
    stats_->launches = launches_;
    stats_->tile_ms = timer_.total_ms();
  }
  return finish(info);
}

}  // namespace

size_t grid_ws_bytes(int kind, bool cplx, int precision, int d, int m) {
  return layout(kind, cplx, precision, d, m).total;
}

int grid_run(const GridJob& g, char* msg, size_t msglen) {
  if (g.cplx) {
    Runner<zd> r(g, msg, msglen);
    return r.run();
  }
  Runner<double> r(g, msg, msglen);
  return r.run();
}

}  // namespace fmk
