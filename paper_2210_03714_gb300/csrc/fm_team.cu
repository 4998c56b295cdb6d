// fm_team.cu -- exp(tA) of one matrix of small order (d <= 512) with every
// step spread over many SMs: one cooperative launch of G thread blocks, the
// steps separated by grid-wide barriers.  The paper's parallel scheme (Sec. 2:
// each (I - c_i B)^{-1} on its own processor, then one sum) maps to
//   a1/a2  B = tA (all blocks), eta = ||tA||_1 and s (every block, the same
//          column sums in the same order), B = tA / 2^s
//   a3     B^2 (when a quadratic system or a d2 term needs it) as 8 x 8 output
//          tiles over all blocks; each M_i = I - c_i B (or I - u1 B - u2 B^2)
//          and its right-hand side element-wise over all blocks; then block i
//          factors M_i (LU with partial pivoting), the systems at once
//   a4     the d right-hand-side columns of every system in column blocks over
//          all blocks (triangular solves with M_i's factors)
//   a6     F = a0 I + d1 B + d2 B^2 + sum_i (weighted) Y_i, element-wise, the
//          systems added in ascending order
//   a7     s squarings F <- F F, each as 8 x 8 tiles over all blocks
// All arithmetic in double on the FP64 pipe; the element-wise steps, the
// factorization and the order of the sums follow the one-CTA kernels, so the
// only differences against them are the association of the products' dot
// products (four interleaved partial sums per output) and of the solves.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/fm.h"
#include "cta_la.cuh"
#include "fm_kernels.cuh"
#include "fm_team.h"

namespace fmk {
namespace {

// barrier state, status and the factorizations' results
struct TeamCtl {
  unsigned count, gen;
  int err;    // a barrier wait ran out: every block stops, the call reports -7
  int bad;    // a non-finite entry of A (or t)
  int info;   // written by block 0 at the end
  int s;
  int fi[kMaxTerms];
};

constexpr int TT8 = 8;  // product tiles: 8 x 8 outputs, four threads per output

template <class T>
struct TeamArgs {
  const T* A;
  int lda;
  double t;
  T* Fout;
  int ldf;
  int n;
  int form;
  double anorm;
  int s_fixed;
  int cw;  // right-hand-side columns per solve item
  T *B, *B2, *F, *P, *LU, *X;
  int* piv;
  TeamCtl* ctl;
};

// Grid-wide barrier of a cooperative launch: thread 0 of each block arrives on
// count; the last one resets it and advances gen, the others wait for gen to
// move.  The wait is bounded (about 2 s of clock cycles): on a timeout the
// block sets err and every block stops at its next barrier.
__device__ bool team_sync(TeamCtl* ctl) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &ctl->gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&ctl->count, 1u) == gridDim.x - 1) {
      atomicExch(&ctl->count, 0u);
      __threadfence();
      atomicAdd(&ctl->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > oz::WAIT) {
          atomicOr(&ctl->err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)&ctl->err == 0;
}

template <class T> __device__ __forceinline__ T shfl_down(T v, int o);
template <> __device__ __forceinline__ double shfl_down<double>(double v, int o) {
  return __shfl_down_sync(0xffffffffu, v, o);
}
template <> __device__ __forceinline__ zd shfl_down<zd>(zd v, int o) {
  return {__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o)};
}

// Output tile (r0, c0) (8 x 8) of P = X Y, all n x n with leading dimension n
// (P: ldp).  Rows r0.. of X and columns c0.. of Y are staged in shared memory
// (sx: 8 x n, sy: n x 8); thread 4o + p sums k = p, p + 4, ... of output o in
// ascending k, and the four partial sums are added as (s0 + s1) + (s2 + s3).
template <class T>
__device__ void team_tile(int n, const T* X, const T* Y, T* P, int ldp, int r0, int c0, T* sx,
                          T* sy) {
  using TT = Tr<T>;
  const int tid = threadIdx.x;
  for (int e = tid; e < TT8 * n; e += NT) {
    const int i = e / n, k = e % n;
    sx[e] = r0 + i < n ? X[(size_t)(r0 + i) * n + k] : TT::zero();
    const int kk = e / TT8, j = e % TT8;
    sy[e] = c0 + j < n ? Y[(size_t)kk * n + c0 + j] : TT::zero();
  }
  __syncthreads();
  const int o = tid >> 2, p = tid & 3, i = o / TT8, j = o % TT8;
  T acc = TT::zero();
  for (int k = p; k < n; k += 4) TT::mac(acc, sx[i * n + k], sy[k * TT8 + j]);
  T w = shfl_down<T>(acc, 1);
  if ((p & 1) == 0) acc = TT::add(acc, w);
  w = shfl_down<T>(acc, 2);
  if (p == 0) {
    acc = TT::add(acc, w);
    if (r0 + i < n && c0 + j < n) P[(size_t)(r0 + i) * ldp + c0 + j] = acc;
  }
  __syncthreads();
}

// P = X Y over the grid: tile t to block t mod G
template <class T>
__device__ void team_prod(int n, const T* X, const T* Y, T* P, int ldp, T* sx, T* sy) {
  const int nt = (n + TT8 - 1) / TT8;
  for (int t = blockIdx.x; t < nt * nt; t += gridDim.x)
    team_tile<T>(n, X, Y, P, ldp, (t / nt) * TT8, (t % nt) * TT8, sx, sy);
}

template <class T>
__global__ void __launch_bounds__(NT, 1) team_expm(TeamArgs<T> a, FmCoef cf) {
  using TT = Tr<T>;
  using R = typename TT::R;
  extern __shared__ __align__(16) char smem[];
  __shared__ __align__(16) Sys s_plan[kMaxTerms];
  __shared__ double s_base[2];
  __shared__ int s_nsys;
  __shared__ R s_red[32];
  const int n = a.n, tid = threadIdx.x, G = gridDim.x;
  const size_t nn = (size_t)n * n;
  const size_t g0 = (size_t)blockIdx.x * NT + tid, gs = (size_t)G * NT;
  TeamCtl* ctl = a.ctl;
  T* sx = (T*)smem;
  T* sy = sx + (size_t)TT8 * n;
  if (tid == 0) s_nsys = plan_systems(cf, a.form, true, s_plan, s_base);

  // a1: B = t A and finiteness
  int bad = !isfinite(a.t);
  for (size_t e = g0; e < nn; e += gs) {
    const T v = a.A[(e / n) * (size_t)a.lda + e % n];
    bad |= !TT::finite(v);
    a.B[e] = TT::rscale(v, a.t);
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(&ctl->bad, 1);
  if (!team_sync(ctl)) return;
  // eta = ||tA||_1 in every block (column sums, rows ascending), s
  R cmax = 0;
  for (int c = tid; c < n; c += NT) {
    R s = 0;
    for (int r = 0; r < n; ++r) s += tmag(a.B[(size_t)r * n + c]);
    cmax = (s > cmax || isnan(s)) ? s : cmax;
  }
  cmax = cta_max<R>(cmax, s_red);
  int info = *(volatile int*)&ctl->bad ? -2 : 0;
  const double eta = a.anorm > 0 ? a.anorm * fabs(a.t) : (double)cmax;
  const int s = a.s_fixed >= 0 ? a.s_fixed : (a.s_fixed == kSRfun ? 0 : select_s(eta, cf.theta));
  for (size_t e = g0; e < nn; e += gs) a.B[e] = tscale(a.B[e], s);
  if (!team_sync(ctl)) return;

  const int nsys = s_nsys;
  bool any_quad = false;
  for (int q = 0; q < nsys; ++q) any_quad |= s_plan[q].quad != 0;
  const bool need_b2 = cf.d2[0] != 0 || any_quad;
  const bool hyb = cf.d1[0] != 0 || cf.d2[0] != 0;
  if (need_b2) {
    team_prod<T>(n, a.B, a.B, a.B2, n, sx, sy);
    if (!team_sync(ctl)) return;
  }
  // F = base I (+ d1 B + d2 B^2); each system's M (into its LU slot) and
  // right-hand side (into its X slot), as the one-CTA kernels form them
  for (size_t e = g0; e < nn; e += gs) {
    const int r = (int)(e / n), c = (int)(e % n);
    T v = TT::rscale(tdiag<T>(r, c), s_base[0]);
    if (hyb) {
      if (cf.d1[0] != 0) v = TT::add(v, TT::rscale(a.B[e], cf.d1[0]));
      if (cf.d2[0] != 0) v = TT::add(v, TT::rscale(a.B2[e], cf.d2[0]));
    }
    a.F[e] = v;
    if (info != 0) continue;
    for (int q = 0; q < nsys; ++q) {
      const Sys& S = s_plan[q];
      T* LUq = a.LU + q * nn;
      T* Xq = a.X + q * nn;
      if (S.quad) {
        T cv = wmul<T>(S.u2r, S.u2i, a.B2[e]);
        if (!(S.u1r == 0.0 && S.u1i == 0.0)) cv = TT::add(wmul<T>(S.u1r, S.u1i, a.B[e]), cv);
        LUq[e] = TT::sub(tdiag<T>(r, c), cv);
        T x = wmul<T>(S.ar[0], S.ai[0], a.B[e]);
        if (S.br[0] != 0.0 || S.bi[0] != 0.0) x = TT::add(x, wmul<T>(S.br[0], S.bi[0], a.B2[e]));
        if (r == c && (S.gr[0] != 0.0 || S.gi[0] != 0.0))
          x = TT::add(x, wmul<T>(S.gr[0], S.gi[0], TT::one()));
        Xq[e] = x;
      } else {
        const T cv = wmul<T>(S.cr, S.ci, a.B[e]);
        LUq[e] = TT::sub(tdiag<T>(r, c), cv);
        Xq[e] = a.form == 1 ? tdiag<T>(r, c) : cv;
      }
    }
  }
  if (!team_sync(ctl)) return;

  if (info == 0 && nsys > 0) {
    // a3: system q factored by block q (mod G)
    for (int q = blockIdx.x; q < nsys; q += G) {
      const int fi = cta_getrf<T, 16>(n, a.LU + q * nn, n, a.piv + q * n, (T*)smem);
      if (tid == 0) ctl->fi[q] = fi;
    }
    if (!team_sync(ctl)) return;
    for (int q = 0; q < nsys; ++q) {
      const int fi = *(volatile int*)&ctl->fi[q];
      if (fi) {
        info = s_plan[q].node * n + fi;
        break;
      }
    }
  }
  if (info == 0 && nsys > 0) {
    // a4: column blocks of every system's right-hand side, solved in place
    const int nb = (n + a.cw - 1) / a.cw;
    for (int it = blockIdx.x; it < nsys * nb; it += G) {
      const int q = it / nb, c0 = (it % nb) * a.cw;
      const int m = a.cw < n - c0 ? a.cw : n - c0;
      cta_getrs_ll<T>(n, a.LU + q * nn, n, a.piv + q * n, m, a.X + q * nn + c0, n, (T*)smem);
    }
    if (!team_sync(ctl)) return;
    // a6: F += Y_q (quadratic systems carry their weights in the right-hand
    // side) or w_q Y_q, ascending q
    for (size_t e = g0; e < nn; e += gs) {
      T v = a.F[e];
      for (int q = 0; q < nsys; ++q) {
        const Sys& S = s_plan[q];
        const T y = a.X[q * nn + e];
        v = S.quad ? TT::add(v, y) : TT::add(v, wmul<T>(S.wr[0], S.wi[0], y));
      }
      a.F[e] = v;
    }
    if (!team_sync(ctl)) return;
  }
  // a7: s squarings, ping-pong between F and P
  T* Fc = a.F;
  T* Pc = a.P;
  if (info == 0) {
    for (int q = 0; q < s; ++q) {
      team_prod<T>(n, Fc, Fc, Pc, n, sx, sy);
      if (!team_sync(ctl)) return;
      T* tmp = Fc;
      Fc = Pc;
      Pc = tmp;
    }
  }
  if (a.s_fixed == kSRfun && info == 0 && !(eta <= cf.theta)) info = -5;
  for (size_t e = g0; e < nn; e += gs) a.Fout[(e / n) * (size_t)a.ldf + e % n] = Fc[e];
  if (blockIdx.x == 0 && tid == 0) {
    ctl->info = info;
    ctl->s = s;
  }
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct TeamLay {
  size_t ctl, B, B2, F, P, LU, X, piv, total;
};

TeamLay team_layout(bool cplx, int n, int nsys) {
  const size_t el = cplx ? 16 : 8, nn = (size_t)n * n;
  TeamLay L;
  size_t o = 0;
  L.ctl = o;
  o += up256(sizeof(TeamCtl));
  L.B = o;
  o += up256(nn * el);
  L.B2 = o;
  o += up256(nn * el);
  L.F = o;
  o += up256(nn * el);
  L.P = o;
  o += up256(nn * el);
  L.LU = o;
  o += up256((size_t)nsys * nn * el);
  L.X = o;
  o += up256((size_t)nsys * nn * el);
  L.piv = o;
  o += up256((size_t)nsys * n * 4);
  L.total = o;
  return L;
}

int count_systems(const FmCoef& cf, int form) {
  Sys sys[kMaxTerms];
  double base[2];
  return plan_systems(cf, form, true, sys, base);
}

// dynamic shared memory of one block: the largest of the LU factorization, the
// left-looking solve and the product staging
size_t team_smem(int n, size_t el) {
  const size_t getrf = ((size_t)n * 16 + 2 * GK * GLD) * el + 256;
  const size_t getrs = ((size_t)16 * n + (size_t)NT * 16 + 64) * el;
  const size_t tile = (size_t)2 * TT8 * n * el;
  size_t m = getrf > getrs ? getrf : getrs;
  m = m > tile ? m : tile;
  return m + 256;
}

template <class T>
int team_launch(const TeamJob& j, char* msg, size_t len) {
  const int n = j.n;
  const int nsys = count_systems(j.cf, j.form);
  const TeamLay L = team_layout(j.cplx, n, nsys);
  char* base = (char*)j.ws;
  TeamArgs<T> a;
  a.A = (const T*)j.A;
  a.lda = j.lda;
  a.t = j.t;
  a.Fout = (T*)j.F;
  a.ldf = j.ldf;
  a.n = n;
  a.form = j.form;
  a.anorm = j.anorm;
  a.s_fixed = j.s_fixed;
  a.B = (T*)(base + L.B);
  a.B2 = (T*)(base + L.B2);
  a.F = (T*)(base + L.F);
  a.P = (T*)(base + L.P);
  a.LU = (T*)(base + L.LU);
  a.X = (T*)(base + L.X);
  a.piv = (int*)(base + L.piv);
  a.ctl = (TeamCtl*)(base + L.ctl);
  const size_t smem = team_smem(n, sizeof(T));
  // per device, once: the kernel's shared-memory limit raised to the largest
  // order's need, and one block per SM checked to fit (so any grid up to the
  // SM count is co-resident)
  static std::mutex mu;
  static int ready[64] = {}, sms_of[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    snprintf(msg, len, "team path setup: %s", e != cudaSuccess ? cudaGetErrorString(e) : "device id");
    return FM_ECUDA;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!ready[dev]) {
      const size_t smax = team_smem(kTeamMaxDim, sizeof(T));
      int sms = 1, per_sm = 0, coop = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(team_expm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, team_expm<T>, NT, smax);
      if (e != cudaSuccess) {
        snprintf(msg, len, "team path setup: %s", cudaGetErrorString(e));
        return FM_ECUDA;
      }
      if (!coop || per_sm < 1) {
        snprintf(msg, len, "team path: the device cannot run a cooperative launch of this size");
        return FM_ECUDA;
      }
      sms_of[dev] = sms;
      ready[dev] = 1;
    }
  }
  const int sms = sms_of[dev];
  // blocks: enough for the product tiles and the solve items, at most one per SM
  const int nt = (n + TT8 - 1) / TT8;
  int G = sms;
  if (G > nt * nt && G > 2 * nsys) G = nt * nt > 2 * nsys ? nt * nt : 2 * nsys;
  if (G < 1) G = 1;
  // solve items: about one column block per block of the grid
  const long long cols = (long long)nsys * n;
  a.cw = nsys > 0 ? (int)((cols + G - 1) / G) : n;
  if (a.cw < 1) a.cw = 1;
  e = cudaMemsetAsync(a.ctl, 0, sizeof(TeamCtl), j.st);
  FmCoef cf = j.cf;
  void* args[] = {(void*)&a, (void*)&cf};
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((const void*)team_expm<T>, dim3(G), dim3(NT), args, smem, j.st);
  if (e != cudaSuccess) {
    snprintf(msg, len, "team path launch: %s", cudaGetErrorString(e));
    return FM_ECUDA;
  }
  if (!j.info_host && !j.s_host) return FM_OK;  // no status wanted: stays asynchronous
  TeamCtl h;
  e = cudaMemcpyAsync(&h, a.ctl, sizeof h, cudaMemcpyDeviceToHost, j.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(j.st);
  if (e != cudaSuccess) {
    snprintf(msg, len, "team path: %s", cudaGetErrorString(e));
    return FM_ECUDA;
  }
  if (j.info_host) *j.info_host = h.err ? -7 : h.info;
  if (j.s_host) *j.s_host = h.s;
  return FM_OK;
}

}  // namespace

int team_systems(const FmCoef& cf, int form) { return count_systems(cf, form); }

size_t team_ws_bytes(bool cplx, int n, int nsys) { return team_layout(cplx, n, nsys).total; }

int team_run(const TeamJob& j, char* msg, size_t len) {
  if (j.n < 1 || j.n > kTeamMaxDim) {
    snprintf(msg, len, "team path: d must be in [1, %d]", kTeamMaxDim);
    return FM_ESHAPE;
  }
  if (j.ws_bytes < team_ws_bytes(j.cplx, j.n, count_systems(j.cf, j.form))) {
    snprintf(msg, len, "team path: workspace too small");
    return FM_ENOMEM;
  }
  return j.cplx ? team_launch<zd>(j, msg, len) : team_launch<double>(j, msg, len);
}

}  // namespace fmk
