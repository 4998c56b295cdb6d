// fm_bgrid.cu -- host side of the grid path over a batch: exp(t_b A_b) for
// every matrix of the batch, each step one launch over the whole batch
// (bgrid.cuh), the tensor-core products as one CTA per 128 x 64 output tile
// of every matrix (oz_tiles in batch mode).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/fm.h"
#include "bgrid.cuh"
#include "fm_bgrid.h"
#include "fm_grid.h"

namespace fmk {
namespace {

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Geo {
  std::vector<grid::BMat> mats;
  std::vector<int4> items;
  long long elems = 0;       // sum of d^2
  long long accp = 0;        // accumulator pairs
  long long pxb = 0, pyb = 0;  // plane bytes (all sets)
  long long rows = 0, cols = 0;
};

Geo geometry(bool cplx, int batch, const int* d, const int64_t* off, const int64_t* voff) {
  Geo g;
  g.mats.resize(batch);
  const int parts = cplx ? 2 : 1;
  for (int b = 0; b < batch; ++b) {
    grid::BMat& M = g.mats[b];
    const int n = d[b] > 0 ? d[b] : 0;  // 0: bad order, -1: the other part of a split batch
    M.d = d[b] > 0 ? n : d[b];
    M.mtn = (n + oz::TM - 1) / oz::TM;
    M.ntn = (n + oz::TN - 1) / oz::TN;
    M.kc = (n + grid::GKC - 1) / grid::GKC;
    M.off = g.elems;
    M.uoff = off ? off[b] : 0;
    M.voff = voff ? voff[b] : 0;
    M.px = g.pxb;
    M.py = g.pyb;
    M.acc = g.accp;
    M.eo = (int)g.rows;
    M.fo = (int)g.cols;
    g.elems += (long long)n * n;
    g.pxb += (long long)parts * M.mtn * M.kc * grid::GXST;
    g.pyb += (long long)(cplx ? 3 : 1) * M.ntn * M.kc * grid::GYST;
    g.accp += (long long)parts * M.mtn * oz::TM * M.ntn * oz::TN;
    g.rows += (long long)M.mtn * oz::TM;
    g.cols += (long long)M.ntn * oz::TN;
    for (int p = 0; p < parts; ++p)
      for (int mt = 0; mt < M.mtn; ++mt)
        for (int nt = 0; nt < M.ntn; ++nt) g.items.push_back(make_int4(b, p, mt, nt));
  }
  // the persistent tile kernel deals items round-robin: longest K first
  std::stable_sort(g.items.begin(), g.items.end(), [&](const int4& x, const int4& y) {
    return g.mats[x.x].kc > g.mats[y.x].kc;
  });
  return g;
}

struct Lay {
  size_t mats, items, alive, mask_e, mask_u, mask_s, sbuf, emax, emax4, prev, ctr, act, cont, B,
      B2, B4, B6, pyB, fyB, pxB2, exB2,
      C, Y, E, F, F1, G, pxC, pxG, py, acc, exC, exG, fy, total;
};

Lay carve(const Geo& g, bool cplx, int batch, bool phi) {
  Lay L;
  const size_t elt = cplx ? 16 : 8;
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o += up(b);
    return at;
  };
  L.mats = take(g.mats.size() * sizeof(grid::BMat));
  L.items = take(g.items.size() * sizeof(int4));
  L.alive = take((size_t)batch * 4);
  L.mask_e = take((size_t)batch * 4);
  L.mask_u = take((size_t)batch * 4);
  L.mask_s = take((size_t)batch * 4);
  L.sbuf = take((size_t)batch * 4);
  L.emax = take((size_t)batch * 8);
  L.emax4 = take((size_t)batch * 8);
  L.prev = take((size_t)batch * 8);
  L.ctr = take(64);
  L.act = take((size_t)kMaxTerms * 4);
  L.cont = take((size_t)kMaxTerms * batch * 4);
  L.B = take((size_t)g.elems * elt);
  L.B2 = take((size_t)g.elems * elt);
  L.B4 = take((size_t)g.elems * elt);
  L.B6 = take((size_t)g.elems * elt);
  L.C = take((size_t)g.elems * elt);
  L.Y = take((size_t)g.elems * elt);
  L.E = take((size_t)g.elems * elt);
  L.F = take((size_t)g.elems * elt);
  L.F1 = take(phi ? (size_t)g.elems * elt : 0);
  L.G = take((size_t)(phi ? 2 : 1) * g.elems * elt);
  L.pxC = take((size_t)g.pxb);
  L.pxG = take((size_t)g.pxb);
  L.py = take((size_t)g.pyb);
  L.pyB = take((size_t)g.pyb);
  L.fyB = take((size_t)g.cols * 4);
  L.pxB2 = take((size_t)g.pxb);
  L.exB2 = take((size_t)g.rows * 4);
  L.acc = take((size_t)g.accp * 16);
  L.exC = take((size_t)g.rows * 4);
  L.exG = take((size_t)g.rows * 4);
  L.fy = take((size_t)g.cols * 4);
  L.total = o;
  return L;
}

// device counters
struct Ctr {
  int active;
  int corrections;
  int err;
  int pad;
  double flops;
  unsigned long long emax;  // largest residual entry (bits) of the matrices correcting
  double dflops;
};

template <class T>
class BRunner {
 public:
  BRunner(const BGridJob& j, char* msg, size_t len) : j_(j), msg_(msg), len_(len) {}
  int run();

 private:
  const BGridJob& j_;
  char* msg_;
  size_t len_;
  cudaStream_t st_ = nullptr;
  cudaError_t err_ = cudaSuccess;
  Geo g_;
  Lay L_;
  char* base_ = nullptr;
  grid::BMat* mats_ = nullptr;
  int4* items_ = nullptr;
  int *alive_ = nullptr, *mask_e_ = nullptr, *mask_u_ = nullptr, *mask_s_ = nullptr, *s_ = nullptr;
  unsigned long long* emax_ = nullptr;
  unsigned long long* emax4_ = nullptr;  // largest entry of B^4 per matrix (bits)
  double* prev_ = nullptr;
  dim3 gE_, gR_, gC_;  // grids: element slices, row slices, column slices
  Ctr* ctr_ = nullptr;
  int* act_ = nullptr;   // per system C = u B^2: matrices that go on after step 0
  int* cont_ = nullptr;  // per system and matrix: goes on after step 0
  T *B_ = nullptr, *B2_ = nullptr, *B4_ = nullptr, *B6_ = nullptr, *C_ = nullptr, *Y_ = nullptr, *E_ = nullptr, *F_ = nullptr,
    *F1_ = nullptr, *G_ = nullptr;
  unsigned char *pxC_ = nullptr, *pxG_ = nullptr, *py_ = nullptr;
  unsigned char* pyB_ = nullptr;  // column planes of B (B^2 and every G B)
  int* fyB_ = nullptr;
  unsigned char* pxB2_ = nullptr;  // row planes of B^2 (B^4, and the residuals of C = u B^2)
  int* exB2_ = nullptr;
  long long* acc_ = nullptr;  // exact sums of the products, (hi, lo) per entry
  int *exC_ = nullptr, *exG_ = nullptr, *fy_ = nullptr;
  long long products_ = 0;
  int sms_ = 1;
  TileTimer timer_;

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
  void api(cudaError_t e, const char* where) {
    if (err_ == cudaSuccess && e != cudaSuccess) {
      err_ = e;
      snprintf(msg_, len_, "%s: %s", where, cudaGetErrorString(e));
    }
  }
  Ctr read_ctr() {
    Ctr h;
    memset(&h, 0, sizeof h);
    api(cudaMemcpyAsync(&h, ctr_, sizeof h, cudaMemcpyDeviceToHost, st_), "reading counters");
    api(cudaStreamSynchronize(st_), "stream synchronize");
    return h;
  }

  // Y = (I - C)^-1 C by residual correction from Y = C, for every live matrix:
  // E = C Y + C - Y, then Y = E Y + Y + E (the product at the digit levels
  // its accuracy needs), until the largest residual entry times d is below
  // 2^-30 (then one more correction).  Every iterate is a function of C, so
  // E (I + Y) = (I + Y) E up to rounding and the update converges as the
  // Newton-Schulz step does; in this order both products of a step take Y
  // as the right operand (one column split per step) and E as the left one
  // gets its row planes from its own epilogue.
  // it0 = 1: the first step is done (b_pairs_shared, b_pair_first) and
  // mask_e holds the matrices that go on.
  // ushared != 0: C = ushared B^2 (a shared system), and the residual's
  // product is ushared (B^2 Y) from B^2's own row planes (pxB2_) instead of
  // C Y from planes of C (the same product up to the rounding of C).
  void correct(int dmax, int nb, int it0 = 0, double ushared = 0.0) {
    const int batch = j_.batch;
    if (it0 == 0)
      api(cudaMemcpyAsync(mask_e_, alive_, (size_t)batch * 4, cudaMemcpyDeviceToDevice, st_),
          "mask copy");
    for (int it = it0; err_ == cudaSuccess; ++it) {
      api(cudaMemsetAsync(&ctr_->active, 0, 4, st_), "counter reset");
      grid::Epi e1;
      e1.Z1 = C_;
      e1.b1r = 1.0;
      e1.Z2 = Y_;
      e1.b2r = -1.0;
      if (ushared != 0.0) {
        e1.ar = ushared;
        prod(B2_, pxB2_, exB2_, false, Y_, e1, E_, mask_e_, emax_, 8, pxG_, exG_);
      } else {
        prod(C_, pxC_, exC_, it == it0, Y_, e1, E_, mask_e_, emax_, 8, pxG_, exG_);
      }
      grid::b_flags<<<nb, 256, 0, st_>>>(batch, mats_, emax_, prev_, it, j_.max_iters, mask_e_,
                                         mask_u_, j_.info_dev, &ctr_->active, &ctr_->corrections,
                                         &ctr_->emax);
      check("correction flags");
      const Ctr h = read_ctr();
      if (err_ != cudaSuccess) break;
      // E Y needs an absolute accuracy of about u max|Y| only, and its error is
      // about 2^(14 - 8 Lmax) 8 sqrt(d) max|Y| max|E|: keep the digit-pair
      // levels that bound requires
      double em;
      memcpy(&em, &h.emax, sizeof em);
      int lmax = 8;
      if (em > 0 && em < 1) {
        const double need = 70.0 + 0.5 * log2((double)dmax) + log2(em);
        lmax = (int)ceil(need / 8.0);
        lmax = lmax < 2 ? 2 : (lmax > 8 ? 8 : lmax);
      }
      grid::Epi e2;
      e2.Z1 = Y_;
      e2.b1r = 1.0;
      e2.Z2 = E_;
      e2.b2r = 1.0;
      // rows of E from the residual's epilogue, columns of Y from its product
      prod(E_, pxG_, exG_, false, Y_, e2, Y_, mask_u_, nullptr, lmax, nullptr, nullptr, false);
      api(cudaMemsetAsync(&ctr_->emax, 0, 8, st_), "counter reset");
      if (h.active == 0) break;
    }
  }

  // out = epilogue(X Y) for every matrix with mask[b]; split_x: compute the
  // row planes of X into px (else they are there already); px_next, ex_next:
  // the epilogue also writes the row planes of out there (out is the left
  // operand of the next product); split_y = false: the column planes of Y
  // are those of the last product (same Y, a subset of its matrices)
  void prod(const T* X, unsigned char* px, int* ex, bool split_x, const T* Yp,
            const grid::Epi& e, T* out, const int* mask, unsigned long long* emax,
            int lmax = 8, unsigned char* px_next = nullptr, int* ex_next = nullptr,
            bool split_y = true, int q_next = -1, unsigned char* pyo = nullptr,
            int* fyo = nullptr) {
    if (err_ != cudaSuccess) return;
    // pyo, fyo (nullable): column planes of Y kept elsewhere than py_, fy_
    unsigned char* py = pyo ? pyo : py_;
    int* fy = fyo ? fyo : fy_;
    const int batch = j_.batch;
    const int parts = grid::El<T>::parts;
    if (split_x) {
      grid::b_split_rows<T><<<gR_, NT, 0, st_>>>(mats_, mask, X, px, ex);
      check("row digit planes");
    }
    if (split_y) {
      grid::b_split_cols<T><<<gC_, NT, 0, st_>>>(mats_, mask, Yp, py, fy);
      check("column digit planes");
    }
    grid::OzTiles a;
    memset(&a, 0, sizeof a);
    a.px = px;
    a.py = py;
    a.nparts = parts;
    a.nseg = parts;
    if (parts == 2) {
      a.sx[0][1] = 1; a.sy[0][1] = 2;
      a.sx[1][0] = 0; a.sy[1][0] = 1;
      a.sx[1][1] = 1; a.sy[1][1] = 0;
    }
    a.ksplit = 1;
    a.lmax = lmax;
    a.acc = acc_;
    a.err = &ctr_->err;
    a.items = items_;
    a.mats = mats_;
    a.mask = mask;
    a.store = 1;
    a.flops = &ctr_->flops;
    a.dflops = &ctr_->dflops;
    a.nitems = (int)g_.items.size();
    const int ctas = a.nitems < sms_ ? a.nitems : sms_;  // persistent: one CTA per SM
    timer_.start(st_);
    grid::oz_tiles<<<ctas, grid::GTHREADS, grid::GSMEM + 1024, st_>>>(a);
    timer_.stop(st_);
    check("tensor-core products");
    if (emax) api(cudaMemsetAsync(emax, 0, (size_t)batch * 8, st_), "maximum reset");
    // q_next >= 0: a squaring; its row planes serve only matrices with s > q_next
    grid::b_epilogue<T><<<gR_, NT, 0, st_>>>(mats_, mask, acc_, ex, fy, grid::epi_modes(e), out,
                                             emax, px_next, ex_next,
                                             q_next >= 0 ? s_ : nullptr, q_next);
    check("product epilogue");
    ++products_;
  }
};

template <class T>
int BRunner<T>::run() {
  const BGridJob& j = j_;
  st_ = j.st;
  const int batch = j.batch;
  const bool phi = j.kind == JOB_PHI1 || j.kind == JOB_PHI1MV;
  const bool trig = j.kind == JOB_TRIG;  // cos in F, sin in F1
  const bool two = phi || trig;
  g_ = geometry(j.cplx, batch, j.d_host, j.off_host, j.voff_host);
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev);
    if (sms_ < 1) sms_ = 1;
  }
  L_ = carve(g_, j.cplx, batch, two);
  if (j.ws_bytes < L_.total) {
    snprintf(msg_, len_, "batched grid path: workspace too small");
    return FM_ENOMEM;
  }
  base_ = (char*)j.ws;
  mats_ = (grid::BMat*)(base_ + L_.mats);
  items_ = (int4*)(base_ + L_.items);
  alive_ = (int*)(base_ + L_.alive);
  mask_e_ = (int*)(base_ + L_.mask_e);
  mask_u_ = (int*)(base_ + L_.mask_u);
  mask_s_ = (int*)(base_ + L_.mask_s);
  s_ = j.s_dev ? j.s_dev : (int*)(base_ + L_.sbuf);
  emax_ = (unsigned long long*)(base_ + L_.emax);
  emax4_ = (unsigned long long*)(base_ + L_.emax4);
  prev_ = (double*)(base_ + L_.prev);
  ctr_ = (Ctr*)(base_ + L_.ctr);
  act_ = (int*)(base_ + L_.act);
  cont_ = (int*)(base_ + L_.cont);
  B_ = (T*)(base_ + L_.B);
  B2_ = (T*)(base_ + L_.B2);
  B4_ = (T*)(base_ + L_.B4);
  B6_ = (T*)(base_ + L_.B6);
  C_ = (T*)(base_ + L_.C);
  Y_ = (T*)(base_ + L_.Y);
  E_ = (T*)(base_ + L_.E);
  F_ = (T*)(base_ + L_.F);
  F1_ = two ? (T*)(base_ + L_.F1) : nullptr;
  G_ = (T*)(base_ + L_.G);
  pxC_ = (unsigned char*)(base_ + L_.pxC);
  pxG_ = (unsigned char*)(base_ + L_.pxG);
  py_ = (unsigned char*)(base_ + L_.py);
  pyB_ = (unsigned char*)(base_ + L_.pyB);
  fyB_ = (int*)(base_ + L_.fyB);
  pxB2_ = (unsigned char*)(base_ + L_.pxB2);
  exB2_ = (int*)(base_ + L_.exB2);
  acc_ = (long long*)(base_ + L_.acc);
  exC_ = (int*)(base_ + L_.exC);
  exG_ = (int*)(base_ + L_.exG);
  fy_ = (int*)(base_ + L_.fy);
  {
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
      api(cudaFuncSetAttribute(grid::oz_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               grid::GSMEM + 1024),
          "cudaFuncSetAttribute");
      attr_set[dev] = err_ == cudaSuccess;
    }
  }
  api(cudaMemcpyAsync(mats_, g_.mats.data(), g_.mats.size() * sizeof(grid::BMat),
                      cudaMemcpyHostToDevice, st_),
      "copying the matrix table");
  api(cudaMemcpyAsync(items_, g_.items.data(), g_.items.size() * sizeof(int4),
                      cudaMemcpyHostToDevice, st_),
      "copying the tile table");
  api(cudaMemsetAsync(ctr_, 0, sizeof(Ctr), st_), "counter reset");
  const FmCoef& cf = j.cf;
  const int nb = (batch + 255) / 256;
  int dmax = 1;
  for (int b = 0; b < batch; ++b) dmax = j.d_host[b] > dmax ? j.d_host[b] : dmax;
  gE_ = dim3(batch, (unsigned)(((long long)dmax * dmax + grid::BE - 1) / grid::BE));
  gR_ = dim3(batch, (unsigned)((dmax + grid::RB - 1) / grid::RB));
  gC_ = dim3(batch, (unsigned)((dmax + grid::CB - 1) / grid::CB));
  // the digit planes outside real rows, columns and 8-value groups stay zero
  api(cudaMemsetAsync(pxC_, 0, (size_t)g_.pxb, st_), "plane reset");
  api(cudaMemsetAsync(pxG_, 0, (size_t)g_.pxb, st_), "plane reset");
  api(cudaMemsetAsync(py_, 0, (size_t)g_.pyb, st_), "plane reset");
  api(cudaMemsetAsync(pyB_, 0, (size_t)g_.pyb, st_), "plane reset");
  api(cudaMemsetAsync(pxB2_, 0, (size_t)g_.pxb, st_), "plane reset");

  // a1/a2
  grid::b_prologue<T><<<batch, NT, 0, st_>>>(mats_, (const T*)j.A, j.t_dev, B_, j.anorm, cf.theta,
                                            j.s_fixed, s_, j.info_dev, alive_);
  check("prologue");
  std::vector<int> s_host(batch);
  api(cudaMemcpyAsync(s_host.data(), s_, (size_t)batch * 4, cudaMemcpyDeviceToHost, st_),
      "reading s");
  api(cudaStreamSynchronize(st_), "stream synchronize");
  if (err_ != cudaSuccess) return FM_ECUDA;
  int s_max = 0;
  for (int v : s_host) s_max = v > s_max ? v : s_max;

  // a3-a6 plan: one system per nonzero node; a pair of nodes +c, -c of the
  // roundoff form shares one system I - c^2 B^2, a term of a conjugate-pair set
  // is one real system I - 2 Re(c) B + |c|^2 B^2 (Sec. 1: one product, x^2, and
  // one inverse per pair of roots)
  const int nf = two ? 2 : 1;
  Sys sys[kMaxTerms];
  double base[2];
  const int nsys = plan_systems(cf, j.form, true, sys, base);
  bool any_quad = false;
  for (int q = 0; q < nsys; ++q) {
    any_quad |= sys[q].quad != 0;
    if (sys[q].quad)  // a quadratic system's g I (plain form) joins the multiple of I
      for (int f = 0; f < nf; ++f) base[f] += sys[q].gr[f];
  }
  // systems C = u B^2 with u real (the fused +-c pairs) take their first
  // correction step from B^4 = B^2 B^2 and B^6 = B^4 B^2, formed once: every
  // such system's step-0 decision in one launch, and the systems a matrix
  // finishes at step 0 go straight into F and G in one pass (b_pairs_shared)
  auto shared_ok = [](const Sys& S) {
    return S.quad && S.u1r == 0.0 && S.u1i == 0.0 && S.u2i == 0.0;
  };
  grid::PairsFirst pf;
  memset(&pf, 0, sizeof pf);
  int qidx[kMaxTerms];  // system -> its index in pf (-1: not a shared one)
  for (int q = 0; q < nsys; ++q) {
    qidx[q] = -1;
    if (!shared_ok(sys[q])) continue;
    const int i = pf.nq++;
    qidx[q] = i;
    const double u = sys[q].u2r;
    pf.u[i] = u;
    pf.u2[i] = u * u;
    pf.u3[i] = u * u * u;
    for (int f = 0; f < nf; ++f) {
      pf.yr[f][i] = sys[q].yr[f];
      pf.yi[f][i] = sys[q].yi[f];
      pf.xr[f][i] = sys[q].xr[f];
      pf.xi[f][i] = sys[q].xi[f];
    }
  }
  bool hybrid = false;
  for (int f = 0; f < nf; ++f) hybrid |= cf.d1[f] != 0 || cf.d2[f] != 0;
  // a7 works in the deviation from the identity (E = F - I; Psi = F1 - I for
  // phi_1; X = C - I and S itself for cos and sin): the combination starts
  // from (base - 1) I for those, so it ends in the deviation (every later
  // term is added to it) and no subtraction of I is needed
  const double base_dev[2] = {base[0] - 1.0, phi ? base[1] - 1.0 : base[1]};
  // F_f = base_f I is written by the shared systems' pass when there are
  // such systems and no hybrid terms
  const bool f_in_pairs = pf.nq > 0 && !hybrid;
  // a6 (first part): F_f = base_f I + d1 B + d2 B^2 for each function
  for (int f = 0; f < nf && !f_in_pairs; ++f) {
    grid::b_init_f<T><<<gE_, NT, 0, st_>>>(mats_, alive_, base_dev[f], f ? F1_ : F_);
    check("initial combination");
  }
  const bool need_b2 = cf.d2[0] != 0 || (two && cf.d2[1] != 0) || any_quad;
  if (need_b2) {
    grid::Epi e;
    prod(B_, pxG_, exG_, true, B_, e, B2_, alive_, nullptr, 8, nullptr, nullptr, true, -1, pyB_,
         fyB_);
  }
  for (int f = 0; f < nf; ++f)
    if (cf.d1[f] != 0 || cf.d2[f] != 0) {
      grid::b_hybrid<T><<<gE_, NT, 0, st_>>>(mats_, alive_, cf.d1[f], B_, cf.d2[f],
                                              cf.d2[f] != 0 ? B2_ : nullptr, f ? F1_ : F_);
      check("hybrid terms");
    }

  bool pair_seen = false;
  double asum_r[2] = {0.0, 0.0}, asum_i[2] = {0.0, 0.0};
  int act_host[kMaxTerms] = {};
  if (pf.nq > 0) {
    grid::Epi e;
    prod(B2_, pxB2_, exB2_, true, B2_, e, B4_, alive_, emax4_, 8, pxG_, exG_);
    // B^6 enters only as u^3 B^6 beside u B^2: it needs the absolute accuracy
    // u max|B^2| 2^-53 / u^3, and the digit products' error at level cap L is
    // about 2^(14 - 8L) 8 sqrt(d) max|B^4| max|B^2|.  With s from ||tA||_1,
    // max|B^4| <= ||B||_1^4 <= theta^4, so L >= (70 + log2(sqrt(d) u^2 theta^4)) / 8
    // suffices (the bound the correction update uses, at its a-priori value);
    // with a caller's norm bound or a forced s, every level is kept.
    int l6 = 8;
    if (j_.anorm <= 0 && j_.s_fixed == -1) {
      double u2max = 0;
      for (int i = 0; i < pf.nq; ++i) u2max = pf.u2[i] > u2max ? pf.u2[i] : u2max;
      const double th4 = cf.theta * cf.theta * cf.theta * cf.theta;
      if (u2max > 0 && th4 > 0) {
        const double need = 70.0 + 0.5 * log2((double)dmax) + log2(u2max * th4);
        l6 = (int)ceil(need / 8.0);
        l6 = l6 < 2 ? 2 : (l6 > 8 ? 8 : l6);
      }
    }
    prod(B4_, pxG_, exG_, false, B2_, e, B6_, alive_, nullptr, l6, nullptr, nullptr, false);
    api(cudaMemsetAsync(act_, 0, (size_t)kMaxTerms * 4, st_), "counter reset");
    grid::b_flags0_shared<<<nb, 256, 0, st_>>>(batch, mats_, alive_, emax4_, pf, j_.max_iters,
                                               cont_, j_.info_dev, act_, &ctr_->corrections);
    check("correction flags");
    grid::b_pairs_shared<T><<<gE_, NT, 0, st_>>>(mats_, alive_, cont_, batch, pf, nf,
                                                  f_in_pairs ? 1 : 0, base_dev[0], base_dev[1], B2_, B4_,
                                                  B6_, F_, F1_, G_, G_ + (size_t)g_.elems);
    check("pair combination");
    api(cudaMemcpyAsync(act_host, act_, (size_t)kMaxTerms * 4, cudaMemcpyDeviceToHost, st_),
        "reading counters");
    api(cudaStreamSynchronize(st_), "stream synchronize");
    pair_seen = true;
    for (int i = 0; i < pf.nq; ++i)
      for (int f = 0; f < nf; ++f) {
        asum_r[f] += pf.xr[f][i];
        asum_i[f] += pf.xi[f][i];
      }
  }

  // a3-a6: the shifted systems, ascending first term
  for (int qs = 0; qs < nsys && err_ == cudaSuccess; ++qs) {
    const Sys& S = sys[qs];
    const int i = qidx[qs];
    if (i >= 0) {
      // a shared system: only the matrices that go on after step 0 are left
      if (act_host[i] == 0) continue;
      const int* cq = cont_ + (size_t)i * batch;
      const double u = pf.u[i];
      api(cudaMemcpyAsync(mask_e_, cq, (size_t)batch * 4, cudaMemcpyDeviceToDevice, st_),
          "mask copy");
      grid::b_pair_first<T><<<gE_, NT, 0, st_>>>(mats_, cq, cq, u, pf.u2[i], pf.u3[i], B2_, B4_,
                                                 B6_, C_, Y_);
      check("first correction");
      correct(dmax, nb, 1, u);  // Y = (I - C)^-1 C
      if (err_ != cudaSuccess) break;
      for (int f = 0; f < nf; ++f) {
        grid::b_pair_acc<T><<<gE_, NT, 0, st_>>>(mats_, cq, S.yr[f], S.yi[f], S.xr[f], S.xi[f],
                                                  Y_, 0, f ? F1_ : F_, G_ + (size_t)f * g_.elems);
        check("pair combination");
      }
      continue;
    }
    if (S.quad)  // C = u1 B + u2 B^2
      grid::b_build_shift2<T><<<gE_, NT, 0, st_>>>(mats_, alive_, B_, S.u1r, S.u1i, B2_, S.u2r,
                                                   S.u2i, C_, Y_);
    else
      grid::b_build_shift<T><<<gE_, NT, 0, st_>>>(mats_, alive_, B_, S.cr, S.ci, C_, Y_);
    check("shift");
    correct(dmax, nb);  // Y = (I - C)^-1 C
    if (err_ != cudaSuccess) break;
    for (int f = 0; f < nf; ++f) {
      T* Ff = f ? F1_ : F_;
      if (S.quad) {
        // (I + Y)(g I + a B + b B^2) = g I + y Y + x (I + Y) B with Y = M^-1 - I:
        // F += y Y now (g I is in base), G += x Y, and x B + G B after the last one
        grid::b_pair_acc<T><<<gE_, NT, 0, st_>>>(mats_, alive_, S.yr[f], S.yi[f], S.xr[f], S.xi[f],
                                                  Y_, !pair_seen, Ff, G_ + (size_t)f * g_.elems);
        check("pair combination");
        asum_r[f] += S.xr[f];
        asum_i[f] += S.xi[f];
      } else {
        grid::b_accumulate<T><<<gE_, NT, 0, st_>>>(mats_, alive_, S.wr[f], S.wi[f], Y_,
                                                    j.form == 1, Ff);
        check("combination");
      }
    }
    if (S.quad) pair_seen = true;
  }
  // the pairs' a B + G B: one product per function, F = G B + F + (sum a) B
  for (int f = 0; f < nf && pair_seen && err_ == cudaSuccess; ++f) {
    T* Ff = f ? F1_ : F_;
    grid::Epi e;
    e.Z1 = Ff;
    e.b1r = 1.0;
    e.Z2 = B_;
    e.b2r = asum_r[f];
    e.b2i = asum_i[f];
    // B's column planes from the B^2 product when it ran (else split here once)
    const bool have_b = need_b2 || f > 0;
    prod(G_ + (size_t)f * g_.elems, pxG_, exG_, true, B_, e, Ff, alive_, nullptr, 8, nullptr,
         nullptr, !have_b, -1, pyB_, fyB_);
  }
  if (err_ != cudaSuccess) return FM_ECUDA;

  // a7 in the deviation from the identity, which F (and F1 for phi_1) hold
  // already: E takes F's buffer (F is not needed any more)
  std::swap(E_, F_);
  for (int q = 0; q < s_max; ++q) {
    grid::b_square_mask<<<nb, 256, 0, st_>>>(batch, alive_, s_, q, mask_s_);
    check("squaring mask");
    if (trig) {
      // double angle (Sec. 1): S <- 2 S C = 2S + 2 X S, X <- 2 C^2 - I - I = 4X + 2 X X
      grid::Epi e1;
      e1.ar = 2.0;
      e1.Z1 = F1_;
      e1.b1r = 2.0;
      prod(E_, pxG_, exG_, q == 0, F1_, e1, F1_, mask_s_, nullptr);
      grid::Epi e;
      e.ar = 2.0;
      e.Z1 = E_;
      e.b1r = 4.0;
      prod(E_, pxG_, exG_, false, E_, e, E_, mask_s_, nullptr, 8, pxG_, exG_, true, q + 1);
      continue;
    }
    if (phi) {
      // (Phi, E) <- ((E + I) Phi / 2, E^2):  Psi <- Psi + E/2 + E Psi / 2
      grid::Epi e1;
      e1.ar = 0.5;
      e1.Z1 = F1_;
      e1.b1r = 1.0;
      e1.Z2 = E_;
      e1.b2r = 0.5;
      prod(E_, pxG_, exG_, q == 0, F1_, e1, F1_, mask_s_, nullptr);
    }
    // E <- 2E + E E (the row planes of E are already there for phi_1)
    grid::Epi e;
    e.Z1 = E_;
    e.b1r = 2.0;
    // (after the first squaring the row planes of E come from the last epilogue)
    prod(E_, pxG_, exG_, q == 0 && !phi, E_, e, E_, mask_s_, nullptr, 8, pxG_, exG_, true, q + 1);
  }
  if (j.kind == JOB_EXPM) {
    grid::b_add_identity<T><<<gE_, NT, 0, st_>>>(mats_, alive_, E_, 1.0, (T*)j.F, 1);
    check("output");
  } else if (trig) {
    grid::b_add_identity<T><<<gE_, NT, 0, st_>>>(mats_, alive_, E_, 1.0, (T*)j.F, 1);
    check("output");
    if (j.E) {
      grid::b_add_identity<T><<<gE_, NT, 0, st_>>>(mats_, alive_, F1_, 0.0, (T*)j.E, 1);
      check("output");
    }
  } else {
    if (j.kind == JOB_PHI1) {
      grid::b_add_identity<T><<<gE_, NT, 0, st_>>>(mats_, alive_, F1_, 1.0, (T*)j.F, 1);
      check("output");
      if (j.E) {
        grid::b_add_identity<T><<<gE_, NT, 0, st_>>>(mats_, alive_, E_, 1.0, (T*)j.E, 1);
        check("output");
      }
    } else {  // W = Phi V = V + Psi V
      grid::b_apply<T><<<gR_, NT, 0, st_>>>(mats_, alive_, F1_, (const T*)j.V, j.m, (T*)j.W);
      check("phi_1 action");
    }
  }
  const Ctr h = read_ctr();
  if (err_ != cudaSuccess) return FM_ECUDA;
  if (h.err) {  // a tensor-core wait timed out: every result of the call is invalid
    grid::b_set_info<<<nb, 256, 0, st_>>>(batch, alive_, -7, j.info_dev);
    check("status");
    api(cudaStreamSynchronize(st_), "stream synchronize");
    if (err_ != cudaSuccess) return FM_ECUDA;
  }
  if (j.stats) {
    fm_stats* st = (fm_stats*)j.stats;
    st->products = products_;
    st->product_flops = h.flops;
    st->digit_flops = h.dflops;
    st->corrections = h.corrections;
    st->launches = launches_;
    st->tile_ms = timer_.total_ms();
  }
  return FM_OK;
}

}  // namespace

size_t bgrid_ws_bytes(int kind, bool cplx, int batch, const int* d_host) {
  Geo g = geometry(cplx, batch, d_host, nullptr, nullptr);
  return carve(g, cplx, batch, kind == JOB_PHI1 || kind == JOB_PHI1MV || kind == JOB_TRIG).total;
}

int bgrid_run(const BGridJob& j, char* msg, size_t len) {
  if (j.cplx) {
    BRunner<zd> r(j, msg, len);
    return r.run();
  }
  BRunner<double> r(j, msg, len);
  return r.run();
}

}  // namespace fmk
