// fm_api.cu -- the C ABI (include/fm.h): argument checks, coefficient packing,
// scratch management and kernel launches.  Every numerical step runs in the
// kernels of fm_kernels.cuh; this file only marshals.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fm.h"
#include "fm_band.h"
#include "fm_bgrid.h"
#include "fm_grid.h"
#include "fm_team.h"
#include "fm_job.h"
#include "fm_launch.h"
#include "fm_trid.h"

using namespace fmk;

namespace {

thread_local char g_err[512] = "";
thread_local fm_stats g_stats;

fm_status fail(fm_status s, const char* msg) {
  snprintf(g_err, sizeof g_err, "%s", msg);
  return s;
}

fm_status cuda_fail(cudaError_t e, const char* where) {
  snprintf(g_err, sizeof g_err, "%s: %s", where, cudaGetErrorString(e));
  return FM_ECUDA;
}

// ---- library-managed scratch: one buffer per (device, stream) ---------------
// Calls on one stream run in stream order, so they can share its buffer;
// calls on different streams get different buffers and may overlap.  A buffer
// grows stream-ordered: the old one is released with cudaFreeAsync on its
// stream (after the work already queued there) and the new one taken with
// cudaMallocAsync.  Each buffer has a lock that a call holds from the lookup
// until it has queued its last launch, so host threads sharing a stream take
// turns and never see a buffer freed under them.
struct Scratch {
  std::mutex mu;
  void* p = nullptr;
  size_t bytes = 0;
};
std::mutex g_mu;
std::map<std::pair<int, uintptr_t>, std::unique_ptr<Scratch>> g_bufs;

fm_status get_scratch(size_t need, const fm_opts* o, void** out, cudaStream_t st,
                      std::unique_lock<std::mutex>* hold) {
  if (o && o->workspace) {
    if (o->workspace_bytes < need) return fail(FM_ENOMEM, "opts.workspace is smaller than fm_workspace_size()");
    *out = o->workspace;
    return FM_OK;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  // cudaStreamPerThread names a different stream in every host thread
  static thread_local char per_thread_key;
  const uintptr_t key = st == cudaStreamPerThread ? (uintptr_t)&per_thread_key : (uintptr_t)st;
  Scratch* b;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    std::unique_ptr<Scratch>& slot = g_bufs[std::make_pair(dev, key)];
    if (!slot) slot.reset(new Scratch);
    b = slot.get();
  }
  *hold = std::unique_lock<std::mutex>(b->mu);
  if (b->bytes < need) {
    if (b->p) {
      e = cudaFreeAsync(b->p, st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync of the library scratch");
      b->p = nullptr;
      b->bytes = 0;
    }
    const size_t sz = need + need / 4;
    e = cudaMallocAsync(&b->p, sz, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->p = nullptr;
      return fail(FM_ENOMEM, "cudaMallocAsync of the library scratch failed");
    }
    b->bytes = sz;
  }
  *out = b->p;
  return FM_OK;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int pick_nb(int dmax) { return dmax <= 512 ? 16 : 8; }

// ---- coefficient packing ----------------------------------------------------
fm_status pack_one(const fm_coeffs* cs, int f, bool complex_ok, FmCoef& cf) {
  if (!cs) return fail(FM_EINVAL, "coefficient set is NULL");
  if (cs->k < 1 || cs->k > FM_MAX_TERMS) return fail(FM_EINVAL, "coefficient set: k must be in [1, 16]");
  if (!cs->c_re || !cs->b_re) return fail(FM_EINVAL, "coefficient set: c_re and b_re are required");
  if (cs->conj_pair != 0 && cs->conj_pair != 1) return fail(FM_EINVAL, "coefficient set: conj_pair must be 0 or 1");
  if (f == 1 && cs->conj_pair != cf.conj_pair)
    return fail(FM_EINVAL, "the two coefficient sets must both be conjugate-pair sets or neither");
  if (f == 0) cf.conj_pair = cs->conj_pair;
  for (int i = 0; i < cs->k; ++i) {
    double ci = cs->c_im ? cs->c_im[i] : 0.0, bi = cs->b_im ? cs->b_im[i] : 0.0;
    if (!isfinite(cs->c_re[i]) || !isfinite(ci) || !isfinite(cs->b_re[i]) || !isfinite(bi))
      return fail(FM_EINVAL, "coefficient set: non-finite value");
    if (!complex_ok && !cs->conj_pair && (ci != 0.0 || bi != 0.0))
      return fail(FM_EINVAL, "complex c_i or b_i need the complex (z) entry points");
    if (f == 0) {
      cf.c_re[i] = cs->c_re[i];
      cf.c_im[i] = ci;
    } else if (cf.c_re[i] != cs->c_re[i] || cf.c_im[i] != ci) {
      return fail(FM_EINVAL, "the two coefficient sets must share the same nodes c_i");
    }
    cf.b_re[f][i] = cs->b_re[i];
    cf.b_im[f][i] = bi;
  }
  if (f == 1 && cs->k != cf.k) return fail(FM_EINVAL, "the two coefficient sets must have the same k");
  cf.k = cs->k;
  cf.a0[f] = cs->a0;
  cf.d1[f] = cs->d1;
  cf.d2[f] = cs->d2;
  if (!isfinite(cs->a0) || !isfinite(cs->d1) || !isfinite(cs->d2))
    return fail(FM_EINVAL, "coefficient set: non-finite a0/d1/d2");
  double th = cs->theta;
  if (!(th > 0) || !isfinite(th)) {
    if (fm_theta(cs, f, ldexp(1.0, -53), &th) != FM_OK || !(th > 0))
      return fail(FM_EINVAL, "coefficient set: theta must be positive");
  }
  cf.theta = (f == 0) ? th : fmin(cf.theta, th);
  return FM_OK;
}

// A conjugate-pair set on complex matrices: each term b_i c_i x / (1 - c_i x)
// + conj(b_i) conj(c_i) x / (1 - conj(c_i) x) (the analytic form of 2 Re(...)),
// written out as two terms (one for a real node, with weight 2 Re(b_i)).
fm_status expand_conj(FmCoef& cf) {
  FmCoef o = cf;
  int k = 0;
  for (int i = 0; i < cf.k; ++i) {
    const bool real_node = cf.c_im[i] == 0.0;
    if (k + (real_node ? 1 : 2) > kMaxTerms)
      return fail(FM_EINVAL, "conjugate-pair set: more than 16 terms once written out for complex matrices");
    o.c_re[k] = cf.c_re[i];
    o.c_im[k] = cf.c_im[i];
    for (int f = 0; f < 2; ++f) {
      o.b_re[f][k] = real_node ? 2.0 * cf.b_re[f][i] : cf.b_re[f][i];
      o.b_im[f][k] = real_node ? 0.0 : cf.b_im[f][i];
    }
    ++k;
    if (real_node) continue;
    o.c_re[k] = cf.c_re[i];
    o.c_im[k] = -cf.c_im[i];
    for (int f = 0; f < 2; ++f) {
      o.b_re[f][k] = cf.b_re[f][i];
      o.b_im[f][k] = -cf.b_im[f][i];
    }
    ++k;
  }
  o.k = k;
  o.conj_pair = 0;
  cf = o;
  return FM_OK;
}

fm_status pack(const fm_coeffs* ce, const fm_coeffs* cp, bool complex_ok, int form, FmCoef& cf) {
  memset(&cf, 0, sizeof cf);
  fm_status s = pack_one(ce, 0, complex_ok, cf);
  if (s) return s;
  cf.nfun = 1;
  if (cp) {
    s = pack_one(cp, 1, complex_ok, cf);
    if (s) return s;
    cf.nfun = 2;
  }
  if (cf.conj_pair && complex_ok) {
    s = expand_conj(cf);
    if (s) return s;
  }
  if (form == FM_PLAIN && !cf.conj_pair)
    for (int f = 0; f < cf.nfun; ++f)
      for (int i = 0; i < cf.k; ++i)
        if (cf.b_im[f][i] != 0.0) return fail(FM_EINVAL, "the plain form needs real weights b_i");
  return FM_OK;
}

fm_opts resolve_opts(const fm_opts* o) {
  fm_opts r;
  fm_opts_default(&r);
  if (o) r = *o;
  return r;
}

fm_status check_opts(const fm_opts& o) {
  if (o.precision < FM_FP64 || o.precision > FM_MIXED) return fail(FM_EINVAL, "opts.precision");
  if (o.form != FM_ROUNDOFF && o.form != FM_PLAIN) return fail(FM_EINVAL, "opts.form");
  if (o.max_ir_iters < 0 || o.max_ir_iters > 20) return fail(FM_EINVAL, "opts.max_ir_iters must be in [0, 20]");
  if (!(o.ir_tol >= 0) || !isfinite(o.anorm) || o.anorm < 0) return fail(FM_EINVAL, "opts.ir_tol / opts.anorm");
  if (o.s_fixed > 1000 || o.s_fixed < kSRfun) return fail(FM_EINVAL, "opts.s_fixed");
  if (o.nsteps < 0) return fail(FM_EINVAL, "opts.nsteps");
  if (o.path < FM_PATH_AUTO || o.path > FM_PATH_TEAM) return fail(FM_EINVAL, "opts.path");
  return FM_OK;
}

// element sizes of the working and factorization types
void type_sizes(bool cplx, int precision, size_t& elt, size_t& lelt) {
  elt = cplx ? 16 : 8;
  lelt = precision == FM_FP64 ? elt : elt / 2;
}

size_t smem_for(bool cplx, int nb, int dmax, int precision) {
  return launch_smem(cplx, nb, dmax, uses_tc(cplx, precision));
}

struct Plan {
  int grid;
  int nb;
  size_t smem;
  size_t per_cta;
  size_t header;
  size_t total;
};

Plan make_plan(int kind, bool cplx, int precision, int batch, int dmax, int m, int k, long long nmax) {
  Plan p;
  p.nb = pick_nb(dmax);
  p.smem = smem_for(cplx, p.nb, dmax, precision);
  size_t elt, lelt;
  type_sizes(cplx, precision, elt, lelt);
  int lk = layout_kind(kind);
  p.per_cta =
      fm_align(ws_layout(lk, dmax, m, k, elt, lelt, nmax, uses_tc(cplx, precision)).total);
  int occ = launch_occupancy(cplx, precision, p.nb, p.smem);
  if (occ < 1) occ = 1;
  long long g = (long long)num_sms() * occ;
  if (g > batch) g = batch;
  if (g < 1) g = 1;
  p.grid = (int)g;
  p.header = 256 + fm_align((size_t)batch * 4);
  p.total = p.header + (size_t)p.grid * p.per_cta;
  return p;
}

// Which kernels run a call.  FM_FP64 runs anywhere; FM_FP32_IR (single
// factors + refinement) only on the one-CTA kernels; FM_BF16_IR (tensor-core
// digit products in the correction iteration) only on the grid paths;
// FM_MIXED picks by path (double on the team kernel).  The batched grid path
// takes exp, phi_1 and phi_1 V; the team kernel single-matrix exp.
enum Route { R_CTA = 0, R_GRID = 1, R_BGRID = 2, R_TEAM = 3, R_BAD = -1 };

Route route(int kind, bool single, int dmax, int precision, int path, const char** why) {
  const bool bg_kind = kind == JOB_EXPM || kind == JOB_PHI1 || kind == JOB_PHI1MV || kind == JOB_TRIG;
  *why = "";
  if (kind == JOB_ADJ) return R_CTA;
  if (path == FM_PATH_TEAM) {
    if (!single || kind != JOB_EXPM) {
      *why = "FM_PATH_TEAM takes single-matrix exp (fm_expm, fm_zexpm, fm_rfun) only";
      return R_BAD;
    }
    if (precision == FM_FP32_IR || precision == FM_BF16_IR) {
      *why = "FM_PATH_TEAM computes in double: FM_FP64 or FM_MIXED";
      return R_BAD;
    }
    if (dmax > kTeamMaxDim) {
      *why = "FM_PATH_TEAM takes d <= 512";
      return R_BAD;
    }
    return R_TEAM;
  }
  if (precision == FM_FP32_IR && path == FM_PATH_GRID) {
    *why = "FM_FP32_IR runs on the one-CTA kernels; the grid paths take FM_FP64, FM_BF16_IR or FM_MIXED";
    return R_BAD;
  }
  if (precision == FM_BF16_IR && path == FM_PATH_CTA) {
    *why = "FM_BF16_IR runs on the grid paths; the one-CTA kernels take FM_FP64, FM_FP32_IR or FM_MIXED";
    return R_BAD;
  }
  const bool want_grid = path == FM_PATH_GRID || precision == FM_BF16_IR;
  if (single) {
    if (want_grid) return R_GRID;
    // one small matrix: every step spread over many SMs beats one block
    if (path == FM_PATH_AUTO && kind == JOB_EXPM && dmax <= kTeamMaxDim &&
        (precision == FM_FP64 || precision == FM_MIXED))
      return R_TEAM;
    if (path == FM_PATH_AUTO && dmax > fm_max_dim()) {
      if (precision == FM_FP32_IR) {
        *why = "FM_FP32_IR runs on the one-CTA kernels (d <= fm_max_dim())";
        return R_BAD;
      }
      return R_GRID;
    }
    return R_CTA;
  }
  if (want_grid) {
    if (!bg_kind) {
      *why = "the grid path takes batches of exp, phi_1 (and phi_1 V) and cos/sin only; other batched "
             "jobs run on the one-CTA kernels (FM_PATH_CTA with FM_FP64, FM_FP32_IR or FM_MIXED)";
      return R_BAD;
    }
    return R_BGRID;
  }
  // batches of exp and phi_1 in FM_MIXED with matrices of order 64 and up: the
  // grid path (tensor-core products over the whole batch) is the faster one
  if (path == FM_PATH_AUTO && bg_kind && precision == FM_MIXED && dmax >= 64 && dmax <= fm_max_dim())
    return R_BGRID;
  return R_CTA;
}

struct Call {
  int kind;
  bool cplx;
  const fm_coeffs* ce;
  const fm_coeffs* cp;
  int batch, dmax, m;
  const int* d_dev;
  const int64_t* off;
  const int64_t* voff;
  int d1, lda, ldf, lde, ldv, ldw;
  const double* t_dev;
  double t1;
  const void* A;
  void* F;
  void* E;
  const void* V;
  void* W;
  int* info_dev;
  int* s_dev;
  const long* nsteps_dev;
  long long nsteps_max;
  const double* wbar;
  double* Abar;
  double* vbar;
  int* info_host;
  int* s_host;
  long* n_host;
  // a part of a split batch: only orders in [part_lo, part_hi] (0: no bound);
  // the others are left to the other part, their status untouched
  int part_lo, part_hi;
};

// single matrix over the whole GPU (fm_grid.cu)
fm_status run_grid(const Call& c, const fm_opts& o, cudaStream_t st) {
  const int n = c.d1;
  const bool act = c.kind == JOB_EXPMV || c.kind == JOB_PHI1MV;
  if (act && c.m < 1) return fail(FM_ESHAPE, "m must be >= 1");
  if (!c.A) return fail(FM_EINVAL, "A is NULL");
  if (!act && !c.F) return fail(FM_EINVAL, "output is NULL");
  if (act && (!c.V || !c.W)) return fail(FM_EINVAL, "V / W is NULL");
  if (c.lda < n || (!act && c.ldf < n) || (c.E && c.lde < n) ||
      (act && (c.ldv < c.m || c.ldw < c.m)))
    return fail(FM_ESHAPE, "leading dimension smaller than the row length");
  GridJob g;
  memset(&g, 0, sizeof g);
  fm_status s = pack(c.ce, c.cp, c.cplx, o.form, g.cf);
  if (s) return s;
  g.kind = c.kind;
  g.cplx = c.cplx;
  g.precision = o.precision;
  g.form = o.form;
  g.d = n;
  g.m = c.m;
  g.A = c.A;
  g.lda = c.lda;
  g.t = c.t1;
  g.F = c.F;
  g.ldf = c.ldf;
  g.E = c.E;
  g.lde = c.lde;
  g.V = c.V;
  g.ldv = c.ldv;
  g.W = c.W;
  g.ldw = c.ldw;
  g.anorm = o.anorm;
  g.s_fixed = o.s_fixed;
  g.nsteps = o.nsteps;
  g.max_iters = 40;
  g.st = st;
  g.info_host = c.info_host;
  g.s_host = c.s_host;
  g.n_host = c.n_host;
  g.stats = &g_stats;
  g.ws_bytes = grid_ws_bytes(c.kind, c.cplx, o.precision, n, c.m);
  std::unique_lock<std::mutex> hold;  // the scratch stays ours until the work is queued
  s = get_scratch(g.ws_bytes, &o, &g.ws, st, &hold);
  if (s) return s;
  return (fm_status)grid_run(g, g_err, sizeof g_err);
}

// a batch of exp over the whole GPU (fm_bgrid.cu)
fm_status run_bgrid(const Call& c, const fm_opts& o, cudaStream_t st) {
  if (c.kind != JOB_EXPM && c.kind != JOB_PHI1 && c.kind != JOB_PHI1MV && c.kind != JOB_TRIG)
    return fail(FM_EINVAL, "the grid path takes batches of exp, phi_1 (and phi_1 V) and cos/sin "
                           "only; other batched jobs: FM_PATH_CTA");
  const bool act = c.kind == JOB_PHI1MV;
  if (!c.A || !c.d_dev || !c.off || !c.t_dev || !c.info_dev)
    return fail(FM_EINVAL, "batched calls need A, d_dev, off_dev, t_dev and info_dev");
  if (act ? (!c.V || !c.W || !c.voff || c.m < 1) : !c.F)
    return fail(FM_EINVAL, "output (or V / W / voff_dev / m) missing");
  if (c.dmax < 1 || c.dmax > fm_max_dim()) return fail(FM_ESHAPE, "dmax must be in [1, fm_max_dim()]");
  BGridJob j;
  memset(&j, 0, sizeof j);
  fm_status s = pack(c.ce, c.cp, c.cplx, o.form, j.cf);
  if (s) return s;
  std::vector<int> d(c.batch);
  std::vector<int64_t> off(c.batch), voff(act ? c.batch : 0);
  cudaError_t e = cudaMemcpyAsync(d.data(), c.d_dev, (size_t)c.batch * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(off.data(), c.off, (size_t)c.batch * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && act)
    e = cudaMemcpyAsync(voff.data(), c.voff, (size_t)c.batch * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "reading the batch orders");
  // a matrix whose order is outside [1, dmax] is left out (order 0 in the
  // tables: no tiles, no elements) and gets info = -4, as on the one-CTA path;
  // one that belongs to the other part of a split batch is left out (order -1)
  // without a status
  for (int b = 0; b < c.batch; ++b) {
    if (d[b] < 1 || d[b] > c.dmax) d[b] = 0;
    else if ((c.part_lo > 0 && d[b] < c.part_lo) || (c.part_hi > 0 && d[b] > c.part_hi)) d[b] = -1;
  }
  j.kind = c.kind;
  j.cplx = c.cplx;
  j.form = o.form;
  j.batch = c.batch;
  j.d_host = d.data();
  j.off_host = off.data();
  j.voff_host = act ? voff.data() : nullptr;
  j.m = c.m;
  j.A = c.A;
  j.t_dev = c.t_dev;
  j.F = c.F;
  j.E = c.E;
  j.V = c.V;
  j.W = c.W;
  j.info_dev = c.info_dev;
  j.s_dev = c.s_dev;
  j.anorm = o.anorm;
  j.s_fixed = o.s_fixed;
  j.max_iters = 40;
  j.st = st;
  j.stats = &g_stats;
  j.ws_bytes = bgrid_ws_bytes(c.kind, c.cplx, c.batch, d.data());
  std::unique_lock<std::mutex> hold;  // the scratch stays ours until the work is queued
  s = get_scratch(j.ws_bytes, &o, &j.ws, st, &hold);
  if (s) return s;
  return (fm_status)bgrid_run(j, g_err, sizeof g_err);
}

// ---- autotuned split of batched matrix functions -----------------------
// fm_autotune records, per device and job, the order d* from which the
// batched grid path beats the one-CTA kernels; FM_PATH_AUTO batches in
// FM_MIXED then run orders below d* on the one-CTA kernels and the rest on the
// grid path.  d* <= 1: everything on the grid path.
struct TuneRec {
  bool have[3] = {false, false, false};
  int dstar[3] = {0, 0, 0};
};
std::mutex g_tune_mu;
std::vector<TuneRec> g_tune;
bool g_tune_loaded = false;

int tune_slot(int kind) {
  switch (kind) {
    case JOB_EXPM: return 0;
    case JOB_PHI1: case JOB_PHI1MV: return 1;
    case JOB_TRIG: return 2;
    default: return -1;
  }
}

std::string device_key(int dev) {
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string k = pr.name;
  for (char& ch : k)
    if (ch == ' ' || ch == '|') ch = '_';
  return k;
}

// the table of FM_TUNE_CACHE (lines "device|slot|dstar"), read once
void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("FM_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    fclose(f);
    return;
  }
  if ((int)g_tune.size() < ndev) g_tune.resize(ndev);
  char line[256];
  while (fgets(line, sizeof line, f)) {
    char name[200];
    int slot = -1, dstar = 0;
    if (sscanf(line, "%199[^|]|%d|%d", name, &slot, &dstar) != 3 || slot < 0 || slot > 2) continue;
    for (int dv = 0; dv < ndev; ++dv)
      if (device_key(dv) == name) {
        g_tune[dv].have[slot] = true;
        g_tune[dv].dstar[slot] = dstar;
      }
  }
  fclose(f);
}

// d* for this device and job, or 0 when not tuned
int tuned_dstar(int kind) {
  const int slot = tune_slot(kind);
  if (slot < 0) return 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  if ((int)g_tune.size() <= dev || !g_tune[dev].have[slot]) return 0;
  const int v = g_tune[dev].dstar[slot];
  return v < 1 ? 1 : v;
}

fm_status run_cta(const Call& c, fm_opts o, cudaStream_t st);

// one small matrix over many SMs (fm_team.cu)
fm_status run_team(const Call& c, const fm_opts& o, cudaStream_t st) {
  const int n = c.d1;
  if (n < 1 || n > kTeamMaxDim) return fail(FM_ESHAPE, "d must be in [1, 512] on FM_PATH_TEAM");
  if (!c.A) return fail(FM_EINVAL, "A is NULL");
  if (!c.F) return fail(FM_EINVAL, "output is NULL");
  if (c.lda < n || c.ldf < n) return fail(FM_ESHAPE, "leading dimension smaller than the row length");
  TeamJob j;
  memset(&j, 0, sizeof j);
  fm_status s = pack(c.ce, c.cp, c.cplx, o.form, j.cf);
  if (s) return s;
  j.cplx = c.cplx;
  j.form = o.form;
  j.n = n;
  j.A = c.A;
  j.lda = c.lda;
  j.t = c.t1;
  j.F = c.F;
  j.ldf = c.ldf;
  j.anorm = o.anorm;
  j.s_fixed = o.s_fixed;
  j.st = st;
  j.info_host = c.info_host;
  j.s_host = c.s_host;
  j.ws_bytes = team_ws_bytes(c.cplx, n, team_systems(j.cf, o.form));
  std::unique_lock<std::mutex> hold;  // the scratch stays ours until the work is done
  s = get_scratch(j.ws_bytes, &o, &j.ws, st, &hold);
  if (s) return s;
  g_stats.launches = 1;
  return (fm_status)team_run(j, g_err, sizeof g_err);
}

fm_status run(const Call& c, const fm_opts* optsp, cudaStream_t st) {
  memset(&g_stats, 0, sizeof g_stats);
  fm_opts o = resolve_opts(optsp);
  fm_status s = check_opts(o);
  if (s) return s;
  if (c.kind == JOB_ADJ) o.precision = FM_FP64;
  if (c.batch < 1) return fail(FM_ESHAPE, "batch must be >= 1");
  const bool single = c.d_dev == nullptr && c.kind != JOB_ADJ;
  const char* why = "";
  Route r = route(c.kind, single, c.dmax, o.precision, o.path, &why);
  if (r == R_BAD) return fail(FM_EINVAL, why);
  // batches of matrix functions in FM_MIXED with a tuned split order
  int dstar = 0;
  if (!single && o.path == FM_PATH_AUTO && o.precision == FM_MIXED && !c.cplx &&
      c.dmax <= fm_max_dim() && tune_slot(c.kind) >= 0 && c.part_lo == 0 && c.part_hi == 0)
    dstar = tuned_dstar(c.kind);
  // the kernels see 0 (double) or 1 (single factors / tensor-core products)
  o.precision = o.precision == FM_FP64 ? 0 : 1;
  if (dstar > 0) {
    if (dstar <= 1) return run_bgrid(c, o, st);
    if (dstar > c.dmax) return run_cta(c, o, st);
    Call lo = c, hi = c;
    lo.part_hi = dstar - 1;
    hi.part_lo = dstar;
    s = run_cta(lo, o, st);
    if (s) return s;
    return run_bgrid(hi, o, st);
  }
  if (r == R_BGRID) return run_bgrid(c, o, st);
  if (r == R_GRID && c.dmax >= 1) return run_grid(c, o, st);
  if (r == R_TEAM) return run_team(c, o, st);
  return run_cta(c, o, st);
}

// the one-CTA kernels (o.precision already 0 or 1)
fm_status run_cta(const Call& c, fm_opts o, cudaStream_t st) {
  fm_status s;
  if (c.dmax < 1 || c.dmax > fm_max_dim()) return fail(FM_ESHAPE, "d (or dmax) must be in [1, fm_max_dim()]");
  if ((c.kind == JOB_EXPMV || c.kind == JOB_PHI1MV) && c.m < 1) return fail(FM_ESHAPE, "m must be >= 1");
  if (!c.A) return fail(FM_EINVAL, "A is NULL");
  if ((c.kind == JOB_EXPM || c.kind == JOB_PHI1 || c.kind == JOB_TRIG) && !c.F)
    return fail(FM_EINVAL, "output is NULL");
  if ((c.kind == JOB_EXPMV || c.kind == JOB_PHI1MV || c.kind == JOB_ADJ) && (!c.V || !c.W))
    return fail(FM_EINVAL, "V / W is NULL");
  if (c.d_dev) {
    if (!c.off || !c.t_dev) return fail(FM_EINVAL, "batched calls need off_dev and t_dev");
    if ((c.kind == JOB_EXPMV || c.kind == JOB_PHI1MV || c.kind == JOB_ADJ) && !c.voff)
      return fail(FM_EINVAL, "batched actions need voff_dev");
  } else {
    const int n = c.d1;
    if (c.lda < n || ((c.kind == JOB_EXPM || c.kind == JOB_PHI1 || c.kind == JOB_TRIG) && c.ldf < n) ||
        (c.E && c.lde < n) ||
        ((c.kind == JOB_EXPMV || c.kind == JOB_PHI1MV) && (c.ldv < c.m || c.ldw < c.m)))
      return fail(FM_ESHAPE, "leading dimension smaller than the row length");
    if (!isfinite(c.t1)) {
      // reported per matrix (info = -2) like a non-finite entry
    }
  }
  FmCoef cf;
  s = pack(c.ce, c.cp, c.cplx, o.form, cf);
  if (s) return s;

  // the lower part of a split batch only holds orders up to part_hi
  const int dplan = c.part_hi > 0 && c.part_hi < c.dmax ? c.part_hi : c.dmax;
  Plan p = make_plan(c.kind, c.cplx, o.precision, c.batch, dplan, c.m, cf.k, c.nsteps_max);
  void* ws = nullptr;
  std::unique_lock<std::mutex> hold;  // the scratch stays ours until the work is queued
  s = get_scratch(p.total, &o, &ws, st, &hold);
  if (s) return s;

  FmJob J;
  memset(&J, 0, sizeof J);
  J.kind = c.kind;
  J.precision = o.precision;
  J.form = o.form;
  J.max_ir = o.max_ir_iters;
  J.ir_tol = o.ir_tol;
  J.anorm = o.anorm;
  J.s_fixed = o.s_fixed;
  J.nsteps = o.nsteps;
  J.nsteps_max = c.nsteps_max;
  J.batch = c.batch;
  J.dmax = c.dmax;
  J.m = c.m;
  J.d = c.d_dev;
  J.off = c.off;
  J.voff = c.voff;
  J.d1 = c.d1;
  J.lda = c.lda;
  J.ldf = c.ldf;
  J.lde = c.lde;
  J.ldv = c.ldv;
  J.ldw = c.ldw;
  J.t = c.t_dev;
  J.t1 = c.t1;
  J.A = c.A;
  J.F = c.F;
  J.E = c.E;
  J.V = c.V;
  J.W = c.W;
  J.nsteps_dev = (const long long*)c.nsteps_dev;
  J.wbar = c.wbar;
  J.Abar = c.Abar;
  J.vbar = c.vbar;
  char* base = (char*)ws;
  J.counter = (int*)base;                       // [0] queue head, [1] items, [2] info (single)
  J.order = c.d_dev ? (int*)(base + 256) : nullptr;
  J.ws = base + p.header;
  J.ws_stride = p.per_cta;
  J.smem_avail = p.smem > 2048 ? p.smem - 2048 : 0;
  J.info = c.d_dev ? c.info_dev : (int*)(base + 8);
  J.sN = c.d_dev ? c.s_dev : (int*)(base + 12);

  cudaError_t e;
  if (c.d_dev) {
    e = launch_order(c.d_dev, c.batch, c.dmax, c.part_lo > 0 ? c.part_lo : 1,
                     c.part_hi > 0 ? c.part_hi : c.dmax, (int*)J.order, J.counter, c.info_dev, st);
    if (e != cudaSuccess) return cuda_fail(e, "order kernel launch");
  } else {
    int hdr[4] = {0, 1, 0, 0};
    e = cudaMemcpyAsync(base, hdr, sizeof hdr, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (queue reset)");
  }
  e = launch_persistent(c.cplx, o.precision, p.nb, J, cf, p.grid, p.smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  if (!c.d_dev && (c.info_host || c.s_host || c.n_host)) {
    int hdr[4];
    e = cudaMemcpyAsync(hdr, base, sizeof hdr, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the status");
    if (c.info_host) *c.info_host = hdr[2];
    if (c.s_host) *c.s_host = hdr[3];
    if (c.n_host) *c.n_host = hdr[3];
  }
  return FM_OK;
}

}  // namespace

extern "C" {

void fm_opts_default(fm_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->precision = FM_MIXED;
  o->form = FM_ROUNDOFF;
  o->max_ir_iters = 2;
  o->ir_tol = 1e-8;
  o->anorm = 0.0;
  o->s_fixed = -1;
  o->nsteps = 0;
  o->path = FM_PATH_AUTO;
}

int fm_max_dim(void) { return 1024; }

size_t fm_workspace_size(int job, int batch, int dmax, int m, int k, const fm_opts* opts) {
  fm_opts o = resolve_opts(opts);
  bool cplx = job == FM_JOB_ZEXPM || job == FM_JOB_ZEXPMV;
  int kind = JOB_EXPM;
  long long nmax = 0;
  switch (job) {
    case FM_JOB_EXPM: case FM_JOB_ZEXPM: kind = JOB_EXPM; break;
    case FM_JOB_PHI1: kind = JOB_PHI1; break;
    case FM_JOB_EXPMV: case FM_JOB_ZEXPMV: kind = JOB_EXPMV; break;
    case FM_JOB_PHI1MV: kind = JOB_PHI1MV; break;
    case FM_JOB_EXPMV_ADJ: kind = JOB_ADJ; nmax = o.nsteps > 0 ? o.nsteps : 1; o.precision = FM_FP64; break;
    case FM_JOB_COSSIN: kind = JOB_TRIG; break;
    case FM_JOB_RFUN: kind = JOB_EXPM; break;
    default: return 0;
  }
  if (batch < 1 || dmax < 1 || k < 1 || k > FM_MAX_TERMS) return 0;
  if (o.precision < FM_FP64 || o.precision > FM_MIXED) return 0;
  // batch == 1 sizes the single-matrix calls; batch > 1 the batched ones
  const char* why = "";
  const Route r = route(kind, batch == 1 && kind != JOB_ADJ, dmax, o.precision, o.path, &why);
  const int prec = o.precision == FM_FP64 ? 0 : 1;
  if (r == R_BAD) return 0;
  if (r == R_GRID) return grid_ws_bytes(kind, cplx, prec, dmax, m);
  if (r == R_TEAM) return team_ws_bytes(cplx, dmax, k);
  if (r == R_BGRID) {
    if (dmax > fm_max_dim()) return 0;
    std::vector<int> d(batch, dmax);
    return bgrid_ws_bytes(kind, cplx, batch, d.data());
  }
  if (dmax > fm_max_dim()) return 0;
  return make_plan(kind, cplx, prec, batch, dmax, m, k, nmax).total;
}

fm_status fm_expm(const fm_coeffs* cs, int d, const double* A, int lda, double t, double* F,
                  int ldf, const fm_opts* opts, void* stream, int* info_host, int* s_host) {
  Call c = {};
  c.kind = JOB_EXPM;
  c.ce = cs;
  c.batch = 1;
  c.dmax = d;
  c.d1 = d;
  c.lda = lda;
  c.ldf = ldf;
  c.t1 = t;
  c.A = A;
  c.F = F;
  c.info_host = info_host;
  c.s_host = s_host;
  return run(c, opts, (cudaStream_t)stream);
}

fm_status fm_zexpm(const fm_coeffs* cs, int d, const double* A, int lda, double t, double* F,
                   int ldf, const fm_opts* opts, void* stream, int* info_host, int* s_host) {
  Call c = {};
  c.kind = JOB_EXPM;
  c.cplx = true;
  c.ce = cs;
  c.batch = 1;
  c.dmax = d;
  c.d1 = d;
  c.lda = lda;
  c.ldf = ldf;
  c.t1 = t;
  c.A = A;
  c.F = F;
  c.info_host = info_host;
  c.s_host = s_host;
  return run(c, opts, (cudaStream_t)stream);
}

fm_status fm_phi1(const fm_coeffs* ce, const fm_coeffs* cphi, int d, const double* A, int lda,
                  double t, double* Phi, int ldp, double* E, int lde, const fm_opts* opts,
                  void* stream, int* info_host, int* s_host) {
  Call c = {};
  c.kind = JOB_PHI1;
  c.ce = ce;
  c.cp = cphi;
  if (!cphi) return fail(FM_EINVAL, "phi_1 needs both coefficient sets");
  c.batch = 1;
  c.dmax = d;
  c.d1 = d;
  c.lda = lda;
  c.ldf = ldp;
  c.lde = lde;
  c.t1 = t;
  c.A = A;
  c.F = Phi;
  c.E = E;
  c.info_host = info_host;
  c.s_host = s_host;
  return run(c, opts, (cudaStream_t)stream);
}

static fm_status action1(bool cplx, const fm_coeffs* cs, int d, const double* A, int lda, double t,
                         int m, const double* V, int ldv, double* W, int ldw, const fm_opts* opts,
                         void* stream, int* info_host, long* n_host) {
  Call c = {};
  c.kind = JOB_EXPMV;
  c.cplx = cplx;
  c.ce = cs;
  c.batch = 1;
  c.dmax = d;
  c.m = m;
  c.d1 = d;
  c.lda = lda;
  c.ldv = ldv;
  c.ldw = ldw;
  c.t1 = t;
  c.A = A;
  c.V = V;
  c.W = W;
  c.info_host = info_host;
  c.n_host = n_host;
  return run(c, opts, (cudaStream_t)stream);
}

fm_status fm_expmv(const fm_coeffs* cs, int d, const double* A, int lda, double t, int m,
                   const double* V, int ldv, double* W, int ldw, const fm_opts* opts,
                   void* stream, int* info_host, long* nsteps_host) {
  return action1(false, cs, d, A, lda, t, m, V, ldv, W, ldw, opts, stream, info_host, nsteps_host);
}

fm_status fm_zexpmv(const fm_coeffs* cs, int d, const double* A, int lda, double t, int m,
                    const double* V, int ldv, double* W, int ldw, const fm_opts* opts,
                    void* stream, int* info_host, long* nsteps_host) {
  return action1(true, cs, d, A, lda, t, m, V, ldv, W, ldw, opts, stream, info_host, nsteps_host);
}

fm_status fm_phi1mv(const fm_coeffs* ce, const fm_coeffs* cphi, int d, const double* A, int lda,
                    double t, int m, const double* V, int ldv, double* W, int ldw,
                    const fm_opts* opts, void* stream, int* info_host, int* s_host) {
  if (!cphi) return fail(FM_EINVAL, "phi_1 needs both coefficient sets");
  Call c = {};
  c.kind = JOB_PHI1MV;
  c.ce = ce;
  c.cp = cphi;
  c.batch = 1;
  c.dmax = d;
  c.m = m;
  c.d1 = d;
  c.lda = lda;
  c.ldv = ldv;
  c.ldw = ldw;
  c.t1 = t;
  c.A = A;
  c.V = V;
  c.W = W;
  c.info_host = info_host;
  c.s_host = s_host;
  return run(c, opts, (cudaStream_t)stream);
}

static fm_status batched(int kind, bool cplx, const fm_coeffs* ce, const fm_coeffs* cp, int batch,
                         int dmax, const int* d_dev, const int64_t* off_dev, const double* A,
                         const double* t_dev, int m, const int64_t* voff_dev, const double* V,
                         double* F, double* E, double* W, int* info_dev, int* s_dev,
                         const fm_opts* opts, void* stream) {
  if (!d_dev || !info_dev) return fail(FM_EINVAL, "batched calls need d_dev and info_dev");
  Call c = {};
  c.kind = kind;
  c.cplx = cplx;
  c.ce = ce;
  c.cp = cp;
  c.batch = batch;
  c.dmax = dmax;
  c.m = m;
  c.d_dev = d_dev;
  c.off = off_dev;
  c.voff = voff_dev;
  c.t_dev = t_dev;
  c.A = A;
  c.F = F;
  c.E = E;
  c.V = V;
  c.W = W;
  c.info_dev = info_dev;
  c.s_dev = s_dev;
  return run(c, opts, (cudaStream_t)stream);
}

fm_status fm_expm_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                          const int64_t* off_dev, const double* A, const double* t_dev,
                          double* F, int* info_dev, int* s_dev, const fm_opts* opts,
                          void* stream) {
  return batched(JOB_EXPM, false, cs, nullptr, batch, dmax, d_dev, off_dev, A, t_dev, 0, nullptr,
                 nullptr, F, nullptr, nullptr, info_dev, s_dev, opts, stream);
}

fm_status fm_zexpm_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                           const int64_t* off_dev, const double* A, const double* t_dev,
                           double* F, int* info_dev, int* s_dev, const fm_opts* opts,
                           void* stream) {
  return batched(JOB_EXPM, true, cs, nullptr, batch, dmax, d_dev, off_dev, A, t_dev, 0, nullptr,
                 nullptr, F, nullptr, nullptr, info_dev, s_dev, opts, stream);
}

fm_status fm_phi1_batched(const fm_coeffs* ce, const fm_coeffs* cphi, int batch, int dmax,
                          const int* d_dev, const int64_t* off_dev, const double* A,
                          const double* t_dev, double* Phi, double* E, int* info_dev,
                          int* s_dev, const fm_opts* opts, void* stream) {
  if (!cphi) return fail(FM_EINVAL, "phi_1 needs both coefficient sets");
  return batched(JOB_PHI1, false, ce, cphi, batch, dmax, d_dev, off_dev, A, t_dev, 0, nullptr,
                 nullptr, Phi, E, nullptr, info_dev, s_dev, opts, stream);
}

fm_status fm_expmv_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                           const int64_t* off_dev, const double* A, const double* t_dev, int m,
                           const int64_t* voff_dev, const double* V, double* W, int* info_dev,
                           int* s_dev, const fm_opts* opts, void* stream) {
  return batched(JOB_EXPMV, false, cs, nullptr, batch, dmax, d_dev, off_dev, A, t_dev, m, voff_dev,
                 V, nullptr, nullptr, W, info_dev, s_dev, opts, stream);
}

fm_status fm_zexpmv_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                            const int64_t* off_dev, const double* A, const double* t_dev, int m,
                            const int64_t* voff_dev, const double* V, double* W, int* info_dev,
                            int* s_dev, const fm_opts* opts, void* stream) {
  return batched(JOB_EXPMV, true, cs, nullptr, batch, dmax, d_dev, off_dev, A, t_dev, m, voff_dev,
                 V, nullptr, nullptr, W, info_dev, s_dev, opts, stream);
}

fm_status fm_phi1mv_batched(const fm_coeffs* ce, const fm_coeffs* cphi, int batch, int dmax,
                            const int* d_dev, const int64_t* off_dev, const double* A,
                            const double* t_dev, int m, const int64_t* voff_dev,
                            const double* V, double* W, int* info_dev, int* s_dev,
                            const fm_opts* opts, void* stream) {
  if (!cphi) return fail(FM_EINVAL, "phi_1 needs both coefficient sets");
  return batched(JOB_PHI1MV, false, ce, cphi, batch, dmax, d_dev, off_dev, A, t_dev, m, voff_dev,
                 V, nullptr, nullptr, W, info_dev, s_dev, opts, stream);
}

fm_status fm_cossin(const fm_coeffs* cc, const fm_coeffs* cs, int d, const double* A, int lda,
                    double t, double* C, int ldc, double* S, int lds, const fm_opts* opts,
                    void* stream, int* info_host, int* s_host) {
  if (!cs) return fail(FM_EINVAL, "fm_cossin needs both coefficient sets");
  Call c = {};
  c.kind = JOB_TRIG;
  c.ce = cc;
  c.cp = cs;
  c.batch = 1;
  c.dmax = d;
  c.d1 = d;
  c.lda = lda;
  c.ldf = ldc;
  c.lde = lds;
  c.t1 = t;
  c.A = A;
  c.F = C;
  c.E = S;
  c.info_host = info_host;
  c.s_host = s_host;
  return run(c, opts, (cudaStream_t)stream);
}

fm_status fm_cossin_batched(const fm_coeffs* cc, const fm_coeffs* cs, int batch, int dmax,
                            const int* d_dev, const int64_t* off_dev, const double* A,
                            const double* t_dev, double* C, double* S, int* info_dev, int* s_dev,
                            const fm_opts* opts, void* stream) {
  if (!cs) return fail(FM_EINVAL, "fm_cossin_batched needs both coefficient sets");
  return batched(JOB_TRIG, false, cc, cs, batch, dmax, d_dev, off_dev, A, t_dev, 0, nullptr,
                 nullptr, C, S, nullptr, info_dev, s_dev, opts, stream);
}

// r(tA) with no range reduction: the exp job with s forced to 0 and the
// theta check of kSRfun
static fm_opts rfun_opts(const fm_opts* opts) {
  fm_opts o = resolve_opts(opts);
  o.s_fixed = kSRfun;
  return o;
}

fm_status fm_rfun(const fm_coeffs* cs, int d, const double* A, int lda, double t, double* F,
                  int ldf, const fm_opts* opts, void* stream, int* info_host) {
  fm_opts o = rfun_opts(opts);
  Call c = {};
  c.kind = JOB_EXPM;
  c.ce = cs;
  c.batch = 1;
  c.dmax = d;
  c.d1 = d;
  c.lda = lda;
  c.ldf = ldf;
  c.t1 = t;
  c.A = A;
  c.F = F;
  c.info_host = info_host;
  return run(c, &o, (cudaStream_t)stream);
}

fm_status fm_rfun_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                          const int64_t* off_dev, const double* A, const double* t_dev, double* F,
                          int* info_dev, const fm_opts* opts, void* stream) {
  fm_opts o = rfun_opts(opts);
  return batched(JOB_EXPM, false, cs, nullptr, batch, dmax, d_dev, off_dev, A, t_dev, 0, nullptr,
                 nullptr, F, nullptr, nullptr, info_dev, nullptr, &o, stream);
}

fm_status fm_expmv_adjoint_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                                   const int64_t* off_dev, const double* A, const double* t_dev,
                                   const long* nsteps_dev, const int64_t* voff_dev,
                                   const double* v, const double* wbar, double* W,
                                   double* Abar, double* vbar, int* info_dev,
                                   const fm_opts* opts, void* stream) {
  if (!d_dev || !info_dev || !nsteps_dev || !wbar || !Abar || !vbar)
    return fail(FM_EINVAL, "adjoint: NULL argument");
  fm_opts o = resolve_opts(opts);
  if (o.nsteps <= 0) return fail(FM_EINVAL, "adjoint: opts.nsteps must bound every nsteps_dev[b]");
  if (cs && cs->conj_pair) return fail(FM_EINVAL, "adjoint: the set must have real nodes (conj_pair = 0)");
  Call c = {};
  c.kind = JOB_ADJ;
  c.ce = cs;
  c.batch = batch;
  c.dmax = dmax;
  c.m = 1;
  c.d_dev = d_dev;
  c.off = off_dev;
  c.voff = voff_dev;
  c.t_dev = t_dev;
  c.A = A;
  c.V = v;
  c.W = W;
  c.wbar = wbar;
  c.Abar = Abar;
  c.vbar = vbar;
  c.nsteps_dev = nsteps_dev;
  c.nsteps_max = o.nsteps;
  c.info_dev = info_dev;
  fm_opts o2 = o;
  o2.nsteps = 0;
  o2.precision = FM_FP64;
  return run(c, &o2, (cudaStream_t)stream);
}

fm_status fm_trid_expmv_batched(const fm_coeffs* cs, int batch, int d, const double* dl,
                                const double* dd, const double* du, const double* t_dev,
                                const double* V, double* W, int* info_dev, int* nsteps_dev,
                                const fm_opts* opts, void* stream) {
  memset(&g_stats, 0, sizeof g_stats);
  fm_opts o = resolve_opts(opts);
  fm_status s = check_opts(o);
  if (s) return s;
  if (batch < 1 || d < 1) return fail(FM_ESHAPE, "fm_trid_expmv_batched: batch and d must be >= 1");
  if (!dd || !t_dev || !V || !W || !info_dev || (d > 1 && (!dl || !du)))
    return fail(FM_EINVAL, "fm_trid_expmv_batched: NULL pointer");
  FmCoef cf;
  s = pack(cs, nullptr, false, o.form, cf);
  if (s) return s;
  if (cf.conj_pair)
    return fail(FM_EINVAL, "fm_trid_expmv_batched: conjugate-pair sets are not taken (their real "
                           "systems I - 2 Re(c) B + |c|^2 B^2 are pentadiagonal)");
  int nonzero = 0;
  for (int i = 0; i < cf.k; ++i) nonzero += cf.c_re[i] != 0.0;
  if (!nonzero) return fail(FM_EINVAL, "fm_trid_expmv_batched: the set needs a nonzero node");
  const size_t need = trid_ws_bytes(batch, d, cf.k);
  void* ws = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  std::unique_lock<std::mutex> hold;  // the scratch stays ours until the work is queued
  s = get_scratch(need, &o, &ws, st, &hold);
  if (s) return s;
  TridJob j;
  j.batch = batch;
  j.d = d;
  j.form = o.form;
  j.dl = dl;
  j.dd = dd;
  j.du = du;
  j.t = t_dev;
  j.V = V;
  j.W = W;
  j.info = info_dev;
  j.nsteps = nsteps_dev;
  j.anorm = o.anorm;
  j.nsteps_fixed = o.nsteps;
  j.cf = cf;
  j.ws = ws;
  j.ws_bytes = o.workspace ? o.workspace_bytes : need;
  j.st = st;
  char msg[256];
  const int r = trid_run(j, msg, sizeof msg);
  if (r) return fail((fm_status)r, msg);
  g_stats.launches = 2;
  return FM_OK;
}

fm_status fm_select_batched(const fm_coeffs* cs, const fm_coeffs* cphi, int job, int batch,
                            int dmax, const int* d_dev, const int64_t* off_dev, const double* A,
                            const double* t_dev, long* out_dev, int* info_dev, const fm_opts* opts,
                            void* stream) {
  memset(&g_stats, 0, sizeof g_stats);
  fm_opts o = resolve_opts(opts);
  fm_status s = check_opts(o);
  if (s) return s;
  bool cplx = false;
  int steps = 0;
  switch (job) {
    case FM_JOB_EXPM: case FM_JOB_PHI1: case FM_JOB_PHI1MV: break;
    case FM_JOB_ZEXPM: cplx = true; break;
    case FM_JOB_EXPMV: case FM_JOB_EXPMV_ADJ: steps = 1; break;
    case FM_JOB_ZEXPMV: cplx = true; steps = 1; break;
    default: return fail(FM_EINVAL, "fm_select_batched: unknown job");
  }
  const bool two = job == FM_JOB_PHI1 || job == FM_JOB_PHI1MV;
  if (two && !cphi) return fail(FM_EINVAL, "fm_select_batched: phi_1 needs both coefficient sets");
  if (batch < 1 || dmax < 1) return fail(FM_ESHAPE, "fm_select_batched: batch and dmax must be >= 1");
  if (!d_dev || !off_dev || !A || !t_dev || !out_dev || !info_dev)
    return fail(FM_EINVAL, "fm_select_batched: NULL pointer");
  FmCoef cf;
  s = pack(cs, two ? cphi : nullptr, cplx, o.form, cf);
  if (s) return s;
  const long long fixed = steps ? (long long)o.nsteps : (long long)o.s_fixed;
  static_assert(sizeof(long) == sizeof(long long), "out_dev holds 64-bit values");
  cudaError_t e = launch_select(cplx, d_dev, off_dev, A, t_dev, batch, dmax, o.anorm, cf.theta,
                                steps, fixed, (long long*)out_dev, info_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "fm_select_batched launch");
  g_stats.launches = 1;
  return FM_OK;
}

fm_status fm_band_expmv_batched(const fm_coeffs* cs, int batch, int d, int p,
                                const double* diags, const double* t_dev, const double* V,
                                double* W, int* info_dev, int* nsteps_dev, const fm_opts* opts,
                                void* stream) {
  if (p == 1) {  // the tridiagonal path, on the same layout
    const size_t plane = (size_t)d * (size_t)(batch > 0 ? batch : 0);
    return fm_trid_expmv_batched(cs, batch, d, diags, diags ? diags + plane : nullptr,
                                 diags ? diags + 2 * plane : nullptr, t_dev, V, W, info_dev,
                                 nsteps_dev, opts, stream);
  }
  memset(&g_stats, 0, sizeof g_stats);
  if (p != 2) return fail(FM_EINVAL, "fm_band_expmv_batched: half bandwidth p must be 1 or 2");
  fm_opts o = resolve_opts(opts);
  fm_status s = check_opts(o);
  if (s) return s;
  if (batch < 1 || d < 1) return fail(FM_ESHAPE, "fm_band_expmv_batched: batch and d must be >= 1");
  if (!diags || !t_dev || !V || !W || !info_dev)
    return fail(FM_EINVAL, "fm_band_expmv_batched: NULL pointer");
  FmCoef cf;
  s = pack(cs, nullptr, false, o.form, cf);
  if (s) return s;
  if (cf.conj_pair)
    return fail(FM_EINVAL, "fm_band_expmv_batched: the set must have real nodes (conj_pair = 0)");
  int nonzero = 0;
  for (int i = 0; i < cf.k; ++i) nonzero += cf.c_re[i] != 0.0;
  if (!nonzero) return fail(FM_EINVAL, "fm_band_expmv_batched: the set needs a nonzero node");
  const size_t need = penta_ws_bytes(batch, d, cf.k);
  void* ws = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  std::unique_lock<std::mutex> hold;  // the scratch stays ours until the work is queued
  s = get_scratch(need, &o, &ws, st, &hold);
  if (s) return s;
  PentaJob j;
  j.batch = batch;
  j.d = d;
  j.form = o.form;
  j.diags = diags;
  j.t = t_dev;
  j.V = V;
  j.W = W;
  j.info = info_dev;
  j.nsteps = nsteps_dev;
  j.anorm = o.anorm;
  j.nsteps_fixed = o.nsteps;
  j.cf = cf;
  j.ws = ws;
  j.ws_bytes = o.workspace ? o.workspace_bytes : need;
  j.st = st;
  char msg[256];
  const int r = penta_run(j, msg, sizeof msg);
  if (r) return fail((fm_status)r, msg);
  g_stats.launches = 2;
  return FM_OK;
}

size_t fm_band_workspace_size(int batch, int d, int p, int k) {
  if (k < 1 || k > FM_MAX_TERMS) return 0;
  if (p == 1) return trid_ws_bytes(batch, d, k);
  if (p == 2) return penta_ws_bytes(batch, d, k);
  return 0;
}

fm_status fm_autotune(const fm_coeffs* ce, const fm_coeffs* cp, int job, int dmax,
                      const fm_opts* opts, void* stream, int* dstar_out, double* table_out,
                      int* nprobe_out) {
  memset(&g_stats, 0, sizeof g_stats);
  int kind;
  switch (job) {
    case FM_JOB_EXPM: kind = JOB_EXPM; break;
    case FM_JOB_PHI1: kind = JOB_PHI1; break;
    case FM_JOB_COSSIN: kind = JOB_TRIG; break;
    default: return fail(FM_EINVAL, "fm_autotune: job must be FM_JOB_EXPM, FM_JOB_PHI1 or FM_JOB_COSSIN");
  }
  const bool two = kind != JOB_EXPM;
  if (two && !cp) return fail(FM_EINVAL, "fm_autotune: this job needs both coefficient sets");
  if (dmax < 1 || dmax > fm_max_dim()) return fail(FM_ESHAPE, "fm_autotune: dmax must be in [1, fm_max_dim()]");
  fm_opts base = resolve_opts(opts);
  fm_status s = check_opts(base);
  if (s) return s;
  base.workspace = nullptr;
  base.workspace_bytes = 0;
  cudaStream_t st = (cudaStream_t)stream;
  static const int kProbe[] = {16, 32, 48, 64, 96, 128, 160, 192, 224, 256, 384, 512, 768, 1024};
  std::vector<int> probes;
  for (int d : kProbe)
    if (d <= dmax) probes.push_back(d);
  if (probes.empty()) probes.push_back(dmax);
  std::vector<double> tc(probes.size()), tg(probes.size());
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "fm_autotune: cudaEventCreate");
  fm_status result = FM_OK;
  for (size_t pi = 0; pi < probes.size() && result == FM_OK; ++pi) {
    const int d = probes[pi];
    long long P = (1LL << 22) / ((long long)d * d);
    P = P < 8 ? 8 : (P > 512 ? 512 : P);
    const size_t nn = (size_t)d * d;
    double *A = nullptr, *F = nullptr, *E = nullptr, *t = nullptr;
    int *dd = nullptr, *info = nullptr, *sv = nullptr;
    int64_t* off = nullptr;
    e = cudaMallocAsync((void**)&A, P * nn * 8, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&F, P * nn * 8, st);
    if (e == cudaSuccess && two) e = cudaMallocAsync((void**)&E, P * nn * 8, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&t, P * 8, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&dd, P * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&info, P * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&sv, P * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&off, P * 8, st);
    std::vector<int> hd(P, d);
    std::vector<int64_t> ho(P);
    std::vector<double> ht(P, 1.0);
    for (long long b = 0; b < P; ++b) ho[b] = b * (int64_t)nn;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dd, hd.data(), P * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(off, ho.data(), P * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t, ht.data(), P * 8, cudaMemcpyHostToDevice, st);
    // ||A||_1 about 4 (entries uniform in [-8/d, 8/d)): a few squarings, as in use
    if (e == cudaSuccess) e = launch_probe_fill(A, (long long)(P * nn), 1234567ULL + d, 8.0 / d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      result = cuda_fail(e, "fm_autotune: probe set-up");
    }
    for (int path = 0; path < 2 && result == FM_OK; ++path) {
      fm_opts o = base;
      o.path = path == 0 ? FM_PATH_CTA : FM_PATH_GRID;
      o.precision = path == 0 ? FM_FP32_IR : FM_BF16_IR;
      Call c = {};
      c.kind = kind;
      c.ce = ce;
      c.cp = two ? cp : nullptr;
      c.batch = (int)P;
      c.dmax = d;
      c.d_dev = dd;
      c.off = off;
      c.t_dev = t;
      c.A = A;
      c.F = F;
      c.E = E;
      c.info_dev = info;
      c.s_dev = sv;
      double best = 1e300;
      for (int rep = 0; rep < 3 && result == FM_OK; ++rep) {
        if (rep > 0) cudaEventRecord(e0, st);
        fm_status r = run(c, &o, st);
        if (r != FM_OK) {
          result = r;
          break;
        }
        if (rep > 0) {
          cudaEventRecord(e1, st);
          e = cudaEventSynchronize(e1);
          float ms = 0;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) {
            result = cuda_fail(e, "fm_autotune: timing");
            break;
          }
          best = fmin(best, (double)ms);
        }
      }
      (path == 0 ? tc : tg)[pi] = best * 1000.0 / (double)P;  // microseconds per matrix
    }
    cudaFreeAsync(A, st);
    cudaFreeAsync(F, st);
    if (E) cudaFreeAsync(E, st);
    cudaFreeAsync(t, st);
    cudaFreeAsync(dd, st);
    cudaFreeAsync(info, st);
    cudaFreeAsync(sv, st);
    cudaFreeAsync(off, st);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != FM_OK) return result;
  // d*: the smallest probe from which the grid path is at least as fast at
  // every larger probe (orders below it take the one-CTA kernels)
  size_t i = probes.size();
  while (i > 0 && tg[i - 1] <= tc[i - 1]) --i;
  const int dstar = i == 0 ? 1 : (i == probes.size() ? dmax + 1 : probes[i]);
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    if ((int)g_tune.size() <= dev) g_tune.resize(dev + 1);
    const int slot = tune_slot(kind);
    g_tune[dev].have[slot] = true;
    g_tune[dev].dstar[slot] = dstar;
    const char* path = getenv("FM_TUNE_CACHE");
    if (path && *path) {
      FILE* f = fopen(path, "a");
      if (f) {
        fprintf(f, "%s|%d|%d\n", device_key(dev).c_str(), slot, dstar);
        fclose(f);
      }
    }
  }
  if (dstar_out) *dstar_out = dstar;
  if (nprobe_out) *nprobe_out = (int)probes.size();
  if (table_out)
    for (size_t q = 0; q < probes.size(); ++q) {
      table_out[3 * q] = probes[q];
      table_out[3 * q + 1] = tc[q];
      table_out[3 * q + 2] = tg[q];
    }
  return FM_OK;
}

void fm_autotune_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  g_tune_loaded = false;  // the next batched call reads FM_TUNE_CACHE again
}

size_t fm_trid_workspace_size(int batch, int d, int k) {
  if (k < 1 || k > FM_MAX_TERMS) return 0;
  return trid_ws_bytes(batch, d, k);
}

const char* fm_last_error(void) { return g_err; }

void fm_last_stats(fm_stats* out) {
  if (out) *out = g_stats;
}

const char* fm_version(void) { return "fm 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// fm_expm_noalloc: exp(tA) for one real matrix with no device allocation.
//
// Some callers cannot allocate device memory at all: code running where
// cudaMalloc is forbidden or could deadlock (inside a custom allocator or a
// memory-pool hook), plugins whose host application owns every device byte,
// and setups that must never grow the device footprint after start-up.  For
// them this entry point uses a fixed scratch array that lives in the library
// image itself (a file-scope __device__ array below), the only scratch this
// call uses.  Inputs and outputs are still the caller's device buffers.
//
// The array belongs to the library's device code, which CUDA loads on a
// device when it is first used there (lazy loading, the default): the first
// call on each device loads it (committing the 2 MiB) and looks up its device
// address (cudaGetSymbolAddress) with that device current.  That first call may
// fail with FM_ECUDA if the device is out of memory; make it once per device as
// a warm-up, before any stream capture and outside any code that must not
// allocate.  Later calls allocate nothing.
//
// Limits: d <= FM_NOALLOC_MAX_DIM (128) and the scratch the call needs must fit
// in FM_NOALLOC_SCRATCH_BYTES (2 MiB); larger problems are rejected with
// FM_ESHAPE.  All calls share the one array: calls that overlap on the GPU (two
// streams, or two host threads) race on it and give wrong results; serialize
// them.  It runs the one-CTA kernel only: opts.path = FM_PATH_GRID or
// FM_PATH_TEAM and opts.precision = FM_BF16_IR are rejected with FM_EINVAL.  It is not for host
// functions enqueued on a stream (cudaLaunchHostFunc): CUDA forbids every CUDA
// call there, and this entry point launches kernels.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = (size_t)FM_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices];  // device address of the array, per device

// Once per device, with that device current: the device address of the array.
// In host code the array's name only stands for it; a kernel must receive this
// address instead.
fm_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(FM_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress of the scratch array");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return FM_OK;
}

}  // namespace

extern "C" fm_status fm_expm_noalloc(const fm_coeffs* cs, int d, const double* A, int lda,
                                     double t, double* F, int ldf, const fm_opts* optsp,
                                     void* stream, int* info_host, int* s_host) {
  cudaStream_t st = (cudaStream_t)stream;
  memset(&g_stats, 0, sizeof g_stats);
  fm_opts o = resolve_opts(optsp);
  fm_status s = check_opts(o);
  if (s) return s;
  if (o.path == FM_PATH_GRID || o.path == FM_PATH_TEAM || o.precision == FM_BF16_IR)
    return fail(FM_EINVAL, "fm_expm_noalloc runs on the one-CTA kernel: opts.path must be "
                           "FM_PATH_AUTO or FM_PATH_CTA, opts.precision not FM_BF16_IR");
  o.precision = o.precision == FM_FP64 ? 0 : 1;
  if (d < 1 || d > FM_NOALLOC_MAX_DIM)
    return fail(FM_ESHAPE, "fm_expm_noalloc: d must be in [1, FM_NOALLOC_MAX_DIM = 128]");
  if (!A || !F) return fail(FM_EINVAL, "A or F is NULL");
  if (lda < d || ldf < d) return fail(FM_ESHAPE, "leading dimension smaller than the row length");
  FmCoef cf;
  s = pack(cs, nullptr, false, o.form, cf);
  if (s) return s;
  size_t elt, lelt;
  type_sizes(false, o.precision, elt, lelt);
  const size_t header = 256;
  const size_t per_cta =
      fm_align(ws_layout(JOB_EXPM, d, 0, cf.k, elt, lelt, 0, uses_tc(false, o.precision)).total);
  if (header + per_cta > kNoAllocBytes)
    return fail(FM_ESHAPE, "fm_expm_noalloc: problem needs more scratch than FM_NOALLOC_SCRATCH_BYTES");
  void* ws = nullptr;
  s = noalloc_scratch(&ws);
  if (s) return s;
  char* base = (char*)ws;
  FmJob J;
  memset(&J, 0, sizeof J);
  J.kind = JOB_EXPM;
  J.precision = o.precision;
  J.form = o.form;
  J.max_ir = o.max_ir_iters;
  J.ir_tol = o.ir_tol;
  J.anorm = o.anorm;
  J.s_fixed = o.s_fixed;
  J.batch = 1;
  J.dmax = d;
  J.d1 = d;
  J.lda = lda;
  J.ldf = ldf;
  J.t1 = t;
  J.A = A;
  J.F = F;
  J.counter = (int*)base;  // work-queue head: must start at zero
  J.info = (int*)(base + 8);
  J.sN = (int*)(base + 12);
  J.ws = base + header;
  J.ws_stride = per_cta;
  cudaError_t e = cudaMemsetAsync(base, 0, 16, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (queue reset)");
  const int nb = pick_nb(d);
  const size_t smem = smem_for(false, nb, d, o.precision);
  J.smem_avail = smem > 2048 ? smem - 2048 : 0;
  e = launch_persistent(false, o.precision, nb, J, cf, 1, smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  if (info_host || s_host) {
    int hdr[4];
    e = cudaMemcpyAsync(hdr, base, sizeof hdr, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the status");
    if (info_host) *info_host = hdr[2];
    if (s_host) *s_host = hdr[3];
  }
  return FM_OK;
}
