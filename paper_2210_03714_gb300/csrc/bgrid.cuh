// bgrid.cuh -- the grid path over a batch of matrices: one launch per step
// for every matrix of the batch (one thread block per matrix for the
// elementwise and split steps, one CTA per 128 x 64 output tile for the
// tensor-core products), masked per matrix.
//
// Same method as the single-matrix grid path (fm_grid.cu): s from the norm
// (Sec. 1, 3), each shifted system (I - C) Y = C, C = c_i B, solved by the
// residual-correction iteration Y <- Y + (I + Y)(C - (I - C) Y) until the
// largest residual entry times d falls below 2^-30 (then one more
// correction), F = a0 I + sum_i b_i Y_i (Eq. ParallRoundOff), and s
// squarings of F = I + E as E <- 2E + E E.
#pragma once
#include "fm_job.h"
#include "grid.cuh"

namespace fmk {
namespace grid {


// block-wide maximum with NaN propagation; red: 32 doubles of shared memory
__device__ __forceinline__ double block_max(double m, double* red) {
  for (int o = 16; o; o >>= 1) {
    const double v = __shfl_xor_sync(0xffffffffu, m, o);
    m = (v > m || isnan(v)) ? v : m;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  double r = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = (red[w] > r || isnan(red[w])) ? red[w] : r;
  return r;
}

// Finiteness, |v| and v 2^-s of an entry.  For real entries they are integer
// operations on the bit pattern (the FP64 pipe, the limit of the elementwise
// passes on GB300, is left to the sums): v 2^-s by subtracting s from the
// exponent field when the result stays normal (exactly the product), by the
// multiplication otherwise (zero, subnormal results, inf, NaN).
template <class T> __device__ __forceinline__ bool entry_finite(T a) { return Tr<T>::finite(a); }
template <> __device__ __forceinline__ bool entry_finite<double>(double a) {
  return ((__double_as_longlong(a) >> 52) & 0x7FF) != 0x7FF;
}
template <class T> __device__ __forceinline__ double entry_mag(T a) { return Tr<T>::mag(a); }
template <> __device__ __forceinline__ double entry_mag<double>(double a) {
  return __longlong_as_double(__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFLL);
}
template <class T> __device__ __forceinline__ T entry_pow2(T a, int s, double p2) {
  return Tr<T>::rscale(a, p2);
}
template <> __device__ __forceinline__ double entry_pow2<double>(double a, int s, double p2) {
  const long long bits = __double_as_longlong(a);
  const int E = (int)((bits >> 52) & 0x7FF);
  return (E > s && E != 0x7FF) ? __longlong_as_double(bits - ((long long)s << 52))
                               : __dmul_rn(a, p2);
}

// a1/a2, one block per matrix: B = t A (one rounding), eta = ||tA||_1 (column
// sums, rows ascending, as the one-CTA kernels), s, B <- B / 2^s; info -2 for
// a non-finite entry or t.  alive[b] = 1 unless info = -2.
template <class T>
__global__ void b_prologue(const BMat* mats, const T* A, const double* t, T* B, double anorm,
                           double theta, int s_fixed, int* s_out, int* info, int* alive) {
  __shared__ double red[32];
  const BMat M = mats[blockIdx.x];
  const int n = M.d, tid = threadIdx.x;
  if (n <= 0) {  // order outside [1, dmax] (0), or the other part of a split batch (-1)
    if (tid == 0) {
      if (n == 0) {
        if (s_out) s_out[blockIdx.x] = 0;
        info[blockIdx.x] = -4;
      }
      alive[blockIdx.x] = 0;
    }
    return;
  }
  const T* Ab = A + M.uoff;
  T* Bb = B + M.off;
  const double tb = t[blockIdx.x];
  int bad = !isfinite(tb);
  // eta = ||fl(t A)||_1: column sums of |fl(t a)|, rows ascending (the order
  // of the one-CTA kernels), with the finiteness check; fl(t A) goes to B
  double cmax = 0;
  for (int c = tid; c < n; c += blockDim.x) {
    double sc = 0;
#pragma unroll 8
    for (int r = 0; r < n; ++r) {
      const T a = Ab[(size_t)r * n + c];
      bad |= !entry_finite<T>(a);
      const T v = tb == 1.0 ? a : Tr<T>::rscale(a, tb);  // t = 1: fl(t a) = a
      Bb[(size_t)r * n + c] = v;
      sc += entry_mag<T>(v);
    }
    cmax = (sc > cmax || isnan(sc)) ? sc : cmax;
  }
  bad = __syncthreads_or(bad);
  cmax = block_max(cmax, red);
  const double eta = anorm > 0 ? anorm * fabs(tb) : cmax;
  int s = s_fixed;
  if (s == kSRfun) {
    s = 0;  // r(tA) as it is: no range reduction
  } else if (s < 0) {
    s = 0;
    while (eta > ldexp(theta, s) && s < 1023) ++s;
  }
  // B = fl(t A) 2^-s (the power of two is exact, so the product is the same
  // correctly rounded value as ldexp gives); block_max's barriers order the
  // column loop's stores before these loads
  if (s > 0) {
    const double p2 = ldexp(1.0, -s);
    for (int e = tid; e < n * n; e += blockDim.x) Bb[e] = entry_pow2<T>(Bb[e], s, p2);
  }
  if (tid == 0) {
    if (s_out) s_out[blockIdx.x] = s;
    info[blockIdx.x] = bad ? -2 : ((s_fixed == kSRfun && !(eta <= theta)) ? -5 : 0);
    alive[blockIdx.x] = !bad;
  }
}

// Elementwise and split kernels run on a grid (batch, parts): block (b, y)
// takes the y-th slice of matrix b (BE elements, or RB rows, or CB columns);
// slices past the end of a small matrix return at once.
constexpr int BE = 4096;  // elements per block
constexpr int RB = 32;    // rows per block (row planes, epilogue)
constexpr int CB = 32;    // columns per block (column planes)

#define FM_SLICE(M, count)                                       \
  if (!mask[blockIdx.x]) return;                                 \
  const BMat M = mats[blockIdx.x];                               \
  const size_t e0 = (size_t)blockIdx.y * BE;                     \
  if (e0 >= (count)) return;                                     \
  const size_t e1 = e0 + BE < (count) ? e0 + BE : (count);

// C = c B, Y = C
template <class T>
__global__ void b_build_shift(const BMat* mats, const int* mask, const T* B, double cr,
                              double ci, T* C, T* Y) {
  FM_SLICE(M, (size_t)mats[blockIdx.x].d * mats[blockIdx.x].d)
#pragma unroll 4
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const T v = cmul<T>(cr, ci, B[M.off + e]);
    C[M.off + e] = v;
    Y[M.off + e] = v;
  }
}

// C = u1 B + u2 B2 (each product rounded once; C = u2 B2 when u1 = 0); Y = C
template <class T>
__global__ void b_build_shift2(const BMat* mats, const int* mask, const T* B, double u1r,
                               double u1i, const T* B2, double u2r, double u2i, T* C, T* Y) {
  FM_SLICE(M, (size_t)mats[blockIdx.x].d * mats[blockIdx.x].d)
  const bool one = u1r == 0.0 && u1i == 0.0;
#pragma unroll 4
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    T v = cmul<T>(u2r, u2i, B2[M.off + e]);
    if (!one) v = Tr<T>::add(cmul<T>(u1r, u1i, B[M.off + e]), v);
    C[M.off + e] = v;
    Y[M.off + e] = v;
  }
}

// The first correction step of a system C = u B^2 (u real: a fused +-c pair,
// u = c^2) from powers of B shared by every such system.  From Y = C the
// residual C Y + C - Y is u^2 B^4 and the update E Y + Y + E is
// u^3 B^6 + u B^2 + u^2 B^4 (the same iterate, in the update's order of
// additions).  Y for every live matrix; C = u B^2 only where cont[b] (the
// matrices that go on correcting).
template <class T>
__global__ void b_pair_first(const BMat* mats, const int* mask, const int* cont, double u,
                             double u2, double u3, const T* B2, const T* B4, const T* B6, T* C,
                             T* Y) {
  FM_SLICE(M, (size_t)mats[blockIdx.x].d * mats[blockIdx.x].d)
  const bool wc = cont[blockIdx.x] != 0;
#pragma unroll 4
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const T c = Tr<T>::rscale(B2[M.off + e], u);
    const T p = Tr<T>::rscale(B6[M.off + e], u3);
    Y[M.off + e] = Tr<T>::add(Tr<T>::add(p, c), Tr<T>::rscale(B4[M.off + e], u2));
    if (wc) C[M.off + e] = c;
  }
}

// Every system C_q = u_q B^2 (u_q real) of a call at once: the weights of
// their first iterates (b_pair_first) in both functions.
struct PairsFirst {
  int nq;
  double u[kMaxTerms], u2[kMaxTerms], u3[kMaxTerms];
  double yr[2][kMaxTerms], yi[2][kMaxTerms], xr[2][kMaxTerms], xi[2][kMaxTerms];
};

// The step-0 decision of b_flags for every system q of P and every matrix,
// from the largest entry of u_q^2 B^4 (the first residual): cont[q batch + b]
// = 1 when system q of matrix b goes on correcting; active[q] counts them.
// A non-finite residual sets info -1 (the matrix stops, as in b_flags).
static __global__ void b_flags0_shared(int batch, const BMat* mats, const int* alive,
                                       const unsigned long long* emax4, PairsFirst P,
                                       int max_iters, int* cont, int* info, int* active,
                                       int* corrections) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const double e4 = __longlong_as_double((long long)emax4[b]);
  for (int q = 0; q < P.nq; ++q) {
    int c = 0;
    if (alive[b]) {
      const double em = e4 * P.u2[q];
      if (em == 0.0) {
      } else if (!(em < INFINITY) || max_iters <= 0) {
        if (info[b] == 0) info[b] = -1;
      } else {
        atomicMax(corrections, 1);
        c = !(em * mats[b].d <= 9.313225746154785e-10 /* 2^-30 */);
      }
    }
    cont[(size_t)q * batch + b] = c;
    if (c) atomicAdd(active + q, 1);
  }
}

// acc + (ar + i ai) z with fused multiply-adds (real: ar z + acc)
template <class T> __device__ __forceinline__ T caxpy(T acc, double ar, double ai, T z);
template <> __device__ __forceinline__ double caxpy<double>(double acc, double ar, double,
                                                            double z) {
  return fma(ar, z, acc);
}
template <> __device__ __forceinline__ zd caxpy<zd>(zd acc, double ar, double ai, zd z) {
  return zd{fma(ar, z.x, fma(-ai, z.y, acc.x)), fma(ar, z.y, fma(ai, z.x, acc.y))};
}

// One pass for the systems of P that a matrix finishes at step 0 (cont = 0).
// Their first iterates Y_q = u_q B^2 + u_q^2 B^4 + u_q^3 B^6 (b_pair_first)
// enter F_f += sum_q y_qf Y_q and G_f = sum_q x_qf Y_q (b_pair_acc) as
// polynomials in B^2: F_f += a1 B^2 + a2 B^4 + a3 B^6 with a_k = sum_q y_qf u_q^k
// over the finished systems (likewise G_f with x_qf), formed once per matrix.
// Each Y_q is never stored, and an entry costs three fused multiply-adds per
// sum instead of nine operations per system (FP64 issue is the limit of
// these passes on GB300).  init: F_f starts from base_f I (no hybrid terms)
// instead of being read.  G_f is written for every live matrix (zero when no
// system finished), so the systems that go on correcting add to it later.
template <class T>
__global__ void b_pairs_shared(const BMat* mats, const int* mask, const int* cont, int batch,
                               PairsFirst P, int nf, int init, double base0, double base1,
                               const T* B2, const T* B4, const T* B6, T* F, T* F1, T* G, T* G1) {
  __shared__ double cf[2][2][3][2];  // [function][F, G][power of B^2][re, im]
  FM_SLICE(M, (size_t)mats[blockIdx.x].d * mats[blockIdx.x].d)
  if (threadIdx.x == 0) {
    for (int f = 0; f < 2; ++f)
      for (int w = 0; w < 2; ++w)
        for (int k = 0; k < 3; ++k) cf[f][w][k][0] = cf[f][w][k][1] = 0.0;
    for (int q = 0; q < P.nq; ++q) {
      if (cont[(size_t)q * batch + blockIdx.x]) continue;
      const double uk[3] = {P.u[q], P.u2[q], P.u3[q]};
      for (int f = 0; f < nf; ++f)
        for (int k = 0; k < 3; ++k) {
          cf[f][0][k][0] += P.yr[f][q] * uk[k];
          cf[f][0][k][1] += P.yi[f][q] * uk[k];
          cf[f][1][k][0] += P.xr[f][q] * uk[k];
          cf[f][1][k][1] += P.xi[f][q] * uk[k];
        }
    }
  }
  __syncthreads();
  const int n = M.d;
  const double c00 = cf[0][0][0][0], c01 = cf[0][0][1][0], c02 = cf[0][0][2][0];
  const double g00 = cf[0][1][0][0], g01 = cf[0][1][1][0], g02 = cf[0][1][2][0];
  const double c00i = cf[0][0][0][1], c01i = cf[0][0][1][1], c02i = cf[0][0][2][1];
  const double g00i = cf[0][1][0][1], g01i = cf[0][1][1][1], g02i = cf[0][1][2][1];
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const size_t i = M.off + e;
    const T b2 = B2[i], b4 = B4[i], b6 = B6[i];
    const bool dg = e / n == e % n;
    T f0 = init ? El<T>::make(dg ? base0 : 0.0, 0.0) : F[i];
    f0 = caxpy<T>(caxpy<T>(caxpy<T>(f0, c02, c02i, b6), c01, c01i, b4), c00, c00i, b2);
    T g0 = cmul<T>(g02, g02i, b6);
    g0 = caxpy<T>(caxpy<T>(g0, g01, g01i, b4), g00, g00i, b2);
    F[i] = f0;
    G[i] = g0;
    if (nf == 2) {
      T f1 = init ? El<T>::make(dg ? base1 : 0.0, 0.0) : F1[i];
      f1 = caxpy<T>(caxpy<T>(caxpy<T>(f1, cf[1][0][2][0], cf[1][0][2][1], b6), cf[1][0][1][0],
                             cf[1][0][1][1], b4),
                    cf[1][0][0][0], cf[1][0][0][1], b2);
      T g1 = cmul<T>(cf[1][1][2][0], cf[1][1][2][1], b6);
      g1 = caxpy<T>(caxpy<T>(g1, cf[1][1][1][0], cf[1][1][1][1], b4), cf[1][1][0][0],
                    cf[1][1][0][1], b2);
      F1[i] = f1;
      G1[i] = g1;
    }
  }
}

// F = base I
template <class T>
__global__ void b_init_f(const BMat* mats, const int* mask, double base, T* F) {
  FM_SLICE(M, (size_t)mats[blockIdx.x].d * mats[blockIdx.x].d)
  const int n = M.d;
#pragma unroll 4
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x)
    F[M.off + e] = Tr<T>::rscale((e / n == e % n) ? Tr<T>::one() : Tr<T>::zero(), base);
}

// F += d1 B + d2 B2 (B2 nullable when d2 == 0)
template <class T>
__global__ void b_hybrid(const BMat* mats, const int* mask, double d1, const T* B, double d2,
                         const T* B2, T* F) {
  FM_SLICE(M, (size_t)mats[blockIdx.x].d * mats[blockIdx.x].d)
#pragma unroll 4
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    T v = F[M.off + e];
    if (d1 != 0) v = Tr<T>::add(v, Tr<T>::rscale(B[M.off + e], d1));
    if (d2 != 0) v = Tr<T>::add(v, Tr<T>::rscale(B2[M.off + e], d2));
    F[M.off + e] = v;
  }
}

// a fused +-c pair with Y = (I - c^2 B^2)^-1 - I:
//   (I + Y)(a B + b' B^2) = a B + a Y B + (b'/c^2) Y,  a = (b+ - b-) c, b'/c^2 = b+ + b-
// F += (b+ + b-) Y here and G += a Y (G = a Y for the first pair); the terms
// a B and G B are added once, after the last pair, by one product
template <class T>
__global__ void b_pair_acc(const BMat* mats, const int* mask, double sr, double si, double ar,
                           double ai, const T* Y, int first, T* F, T* G) {
  FM_SLICE(M, (size_t)mats[blockIdx.x].d * mats[blockIdx.x].d)
#pragma unroll 4
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const T y = Y[M.off + e];
    F[M.off + e] = Tr<T>::add(F[M.off + e], cmul<T>(sr, si, y));
    const T g = cmul<T>(ar, ai, y);
    G[M.off + e] = first ? g : Tr<T>::add(G[M.off + e], g);
  }
}

// F += b Y (roundoff form) or b (I + Y) (plain form)
template <class T>
__global__ void b_accumulate(const BMat* mats, const int* mask, double br, double bi, const T* Y,
                             int plain, T* F) {
  FM_SLICE(M, (size_t)mats[blockIdx.x].d * mats[blockIdx.x].d)
  const int n = M.d;
#pragma unroll 4
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    T y = Y[M.off + e];
    if (plain && e / n == e % n) y = Tr<T>::add(y, Tr<T>::one());
    F[M.off + e] = Tr<T>::add(F[M.off + e], cmul<T>(br, bi, y));
  }
}

// out = in + g I; user_out: out uses the caller's offsets
template <class T>
__global__ void b_add_identity(const BMat* mats, const int* mask, const T* in, double g, T* out,
                               int user_out) {
  FM_SLICE(M, (size_t)mats[blockIdx.x].d * mats[blockIdx.x].d)
  const int n = M.d;
  T* o = out + (user_out ? M.uoff : M.off);
#pragma unroll 4
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    T v = in[M.off + e];
    if (e / n == e % n) v = Tr<T>::add(v, Tr<T>::rscale(Tr<T>::one(), g));
    o[e] = v;
  }
}

// The row digit planes of rows [r0, r0 + nr) of X_b (Xb: its first element,
// d x d) with the rows' exponents s_e (shared memory, set by the caller).
// Only real rows and the 8-value groups holding real columns are written; the
// rest of the planes stays zero from the reset at the start of the call.
template <class T>
__device__ __forceinline__ void row_planes(const BMat& M, const T* Xb, int r0, int nr,
                                           const int* s_e, unsigned char* px) {
  const int n = M.d, kc = M.kc;
  unsigned char* pb = px + M.px;
  const size_t pxs = (size_t)M.mtn * kc * GXST;
  const int g8 = (n + 7) / 8;  // 8-value groups holding real columns
  const int items = nr * g8;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int k8 = it % g8;
    const int rr = it / g8, r = r0 + rr;
    const int e = s_e[rr];
    __align__(16) __nv_bfloat16 dr[oz::S][8], di[oz::S][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k8 * 8 + j;
      const T v = k < n ? Xb[(size_t)r * n + k] : El<T>::make(0.0, 0.0);
      __nv_bfloat16 t[oz::S];
      oz::digits(El<T>::re(v), e, t);
#pragma unroll
      for (int p = 0; p < oz::S; ++p) dr[p][j] = t[p];
      if (El<T>::parts == 2) {
        oz::digits(El<T>::im(v), e, t);
#pragma unroll
        for (int p = 0; p < oz::S; ++p) di[p][j] = t[p];
      }
    }
    const size_t blk = ((size_t)(r / oz::TM) * kc + (k8 * 8) / GKC) * GXST;
    const uint32_t off = plane_off16(r % oz::TM, (k8 * 8) % GKC);
#pragma unroll
    for (int p = 0; p < oz::S; ++p) *(uint4*)(pb + blk + p * GXB + off) = *(const uint4*)dr[p];
    if (El<T>::parts == 2) {
#pragma unroll
      for (int p = 0; p < oz::S; ++p) *(uint4*)(pb + pxs + blk + p * GXB + off) = *(const uint4*)di[p];
    }
  }
}

// Row digit planes of rows [RB y, RB y + RB) of X_b (d x d) and their exponents
// ex[eo + r] (one warp per row for the row's largest entry).
template <class T>
__global__ void b_split_rows(const BMat* mats, const int* mask, const T* X, unsigned char* px,
                             int* ex) {
  __shared__ int s_e[RB];
  if (!mask[blockIdx.x]) return;
  const BMat M = mats[blockIdx.x];
  const int n = M.d;
  const int r0 = blockIdx.y * RB;
  if (r0 >= n) return;
  const int nr = min(RB, n - r0);
  const T* Xb = X + M.off;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int rr = w; rr < nr; rr += nw) {
    const int r = r0 + rr;
    unsigned long long mx = 0;  // largest |re|, |im| as bits: integer operations only
    for (int k = lane; k < n; k += 32) {
      const unsigned long long b = abs_bits<T>(Xb[(size_t)r * n + k]);
      mx = b > mx ? b : mx;
    }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = b > mx ? b : mx;
    }
    if (lane == 0) {
      s_e[rr] = oz::exp_above_bits(mx);
      ex[M.eo + r] = s_e[rr];
    }
  }
  __syncthreads();
  row_planes<T>(M, Xb, r0, nr, s_e, px);
}

// Column digit planes of columns [CB y, CB y + CB) of Y_b (N-major) and their
// exponents fy[fo + j]; only real columns and real 8-value groups of rows.
template <class T>
__global__ void b_split_cols(const BMat* mats, const int* mask, const T* Y, unsigned char* py,
                             int* fy) {
  __shared__ unsigned long long red[8][CB + 1];
  __shared__ int s_f[CB];
  if (!mask[blockIdx.x]) return;
  const BMat M = mats[blockIdx.x];
  const int n = M.d, kc = M.kc;
  const int c0 = blockIdx.y * CB;
  if (c0 >= n) return;
  const int nc = min(CB, n - c0);
  const T* Yb = Y + M.off;
  {
    const int cx = threadIdx.x % CB, ry = threadIdx.x / CB;  // 8 row lanes x 32 columns
    unsigned long long mx = 0;
    if (cx < nc)
      for (int k = ry; k < n; k += 8) {
        const unsigned long long b = abs_bits<T>(Yb[(size_t)k * n + c0 + cx]);
        mx = b > mx ? b : mx;
      }
    red[ry][cx] = mx;
    __syncthreads();
    if (ry == 0) {
      for (int q = 1; q < 8; ++q) mx = red[q][cx] > mx ? red[q][cx] : mx;
      if (cx < nc) {
        s_f[cx] = oz::exp_above_bits(mx);
        fy[M.fo + c0 + cx] = s_f[cx];
      }
    }
    __syncthreads();
  }
  unsigned char* pb = py + M.py;
  const size_t pys = (size_t)M.ntn * kc * GYST;
  const int g8 = (n + 7) / 8;
  const int items = nc * g8;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int jj = it % nc, j = c0 + jj;
    const int k8 = it / nc;
    const int e = s_f[jj];
    __align__(16) __nv_bfloat16 dr[oz::S][8], di[oz::S][8], dn[oz::S][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = k8 * 8 + q;
      const T v = k < n ? Yb[(size_t)k * n + j] : El<T>::make(0.0, 0.0);
      __nv_bfloat16 t[oz::S];
      oz::digits(El<T>::re(v), e, t);
#pragma unroll
      for (int p = 0; p < oz::S; ++p) dr[p][q] = t[p];
      if (El<T>::parts == 2) {
        oz::digits(El<T>::im(v), e, t);
#pragma unroll
        for (int p = 0; p < oz::S; ++p) {
          di[p][q] = t[p];
          dn[p][q] = __hneg(t[p]);
        }
      }
    }
    const size_t blk = ((size_t)(j / oz::TN) * kc + (k8 * 8) / GKC) * GYST;
    const uint32_t off = plane_off16(j % oz::TN, (k8 * 8) % GKC);
#pragma unroll
    for (int p = 0; p < oz::S; ++p) *(uint4*)(pb + blk + p * GYB + off) = *(const uint4*)dr[p];
    if (El<T>::parts == 2) {
#pragma unroll
      for (int p = 0; p < oz::S; ++p) {
        *(uint4*)(pb + pys + blk + p * GYB + off) = *(const uint4*)di[p];
        *(uint4*)(pb + 2 * pys + blk + p * GYB + off) = *(const uint4*)dn[p];
      }
    }
  }
}

// An epilogue's weights with their cases decided on the host, so that the
// element loop runs only the arithmetic each term needs (a test of a double
// weight inside the loop costs an FP64 instruction per element):
//   am      0: alpha = 1, 1: real alpha, 2: complex alpha
//   m1, m2  0: no term, 1: + Z, 2: - Z, 3: + b Z (b real), 4: + b Z (b complex)
//   gd      1: + g on the diagonal
struct EpiModes {
  const void* Z1;
  const void* Z2;
  double ar, ai, b1r, b1i, b2r, b2i, gr, gi;
  int am, m1, m2, gd;
};

inline EpiModes epi_modes(const Epi& e) {
  EpiModes m;
  m.Z1 = e.Z1;
  m.Z2 = e.Z2;
  m.ar = e.ar;
  m.ai = e.ai;
  m.b1r = e.b1r;
  m.b1i = e.b1i;
  m.b2r = e.b2r;
  m.b2i = e.b2i;
  m.gr = e.gr;
  m.gi = e.gi;
  m.am = (e.ar == 1.0 && e.ai == 0) ? 0 : (e.ai == 0 ? 1 : 2);
  auto mode = [](const void* z, double br, double bi) {
    if (!z) return 0;
    if (bi == 0 && br == 1.0) return 1;
    if (bi == 0 && br == -1.0) return 2;
    return bi == 0 ? 3 : 4;
  };
  m.m1 = mode(e.Z1, e.b1r, e.b1i);
  m.m2 = mode(e.Z2, e.b2r, e.b2i);
  m.gd = (e.gr != 0 || e.gi != 0) ? 1 : 0;
  return m;
}

// one weighted term, its case a compile-time constant (1: + Z, 2: - Z, 3: + b Z
// with b real, 4: + b Z with b complex)
template <class T, int M>
__device__ __forceinline__ T epi_term(T v, double br, double bi, T z) {
  if constexpr (M == 1) return Tr<T>::add(v, z);
  else if constexpr (M == 2) return Tr<T>::sub(v, z);
  else if constexpr (M == 3) return Tr<T>::add(v, Tr<T>::rscale(z, br));
  else return Tr<T>::add(v, cmul<T>(br, bi, z));
}

template <class T>
__device__ __forceinline__ T epi_term_rt(T v, int mode, double br, double bi, T z) {
  if (mode == 1) return Tr<T>::add(v, z);
  if (mode == 2) return Tr<T>::sub(v, z);
  if (mode == 3) return Tr<T>::add(v, Tr<T>::rscale(z, br));
  return Tr<T>::add(v, cmul<T>(br, bi, z));
}

// the entries c = lane, lane + 32, ... of one row: P from the exact sums
// (a0: the row's (hi, lo) pairs, part 1 at pst pairs further), the weights'
// cases as template constants (AM < 0, M1 < 0: the cases read at run time,
// with the diagonal term).  Returns the largest |re|, |im| (bits).  Cases
// decided inside the loop would be compiled to predicated instructions of
// every case, each taking an FP64 issue slot per entry.
template <class T, int AM, int M1, int M2>
__device__ __forceinline__ unsigned long long epi_row(const EpiModes& e, const long long* a0,
                                                      size_t pst, int er, const int* fyb,
                                                      const T* z1, const T* z2, T* o, int n,
                                                      int r, int lane) {
  unsigned long long mx = 0;
#pragma unroll 2
  for (int c = lane; c < n; c += 32) {
    const int e2 = er + fyb[c];
    const longlong2 p0 = *(const longlong2*)(a0 + (size_t)c * 2);
    double pi = 0;
    if (El<T>::parts == 2) {
      const longlong2 p1 = *(const longlong2*)(a0 + (pst + c) * 2);
      pi = oz::combine_scaled(p1.x, p1.y, e2);
    }
    T v = El<T>::make(oz::combine_scaled(p0.x, p0.y, e2), pi);
    if constexpr (AM >= 0 && M1 >= 0) {
      if constexpr (AM == 1) v = Tr<T>::rscale(v, e.ar);
      if constexpr (AM == 2) v = cmul<T>(e.ar, e.ai, v);
      if constexpr (M1 > 0) v = epi_term<T, M1>(v, e.b1r, e.b1i, z1[c]);
      if constexpr (M2 > 0) v = epi_term<T, M2>(v, e.b2r, e.b2i, z2[c]);
    } else {
      if (e.am == 1) v = Tr<T>::rscale(v, e.ar);
      else if (e.am == 2) v = cmul<T>(e.ar, e.ai, v);
      if (e.m1) v = epi_term_rt<T>(v, e.m1, e.b1r, e.b1i, z1[c]);
      if (e.m2) v = epi_term_rt<T>(v, e.m2, e.b2r, e.b2i, z2[c]);
      if (e.gd && r == c) v = Tr<T>::add(v, El<T>::make(e.gr, e.gi));
    }
    o[c] = v;
    const unsigned long long b = abs_bits<T>(v);
    mx = b > mx ? b : mx;
  }
  return mx;
}

// rows [RB y, RB y + RB) of out_b = alpha P_b + b1 Z1_b + b2 Z2_b + g I, one
// warp per row; P_b from the exact sums (rounded once).  emax[b] (bits,
// zeroed by the caller, nullable) = largest |re|, |im| of out_b.  px, ex
// (nullable): also the row digit planes of out_b and their exponents, for a
// product that takes out_b as its left operand next (no separate row split).
template <class T>
__global__ void b_epilogue(const BMat* mats, const int* mask, const long long* acc,
                           const int* exs, const int* fy, EpiModes e, T* out,
                           unsigned long long* emax, unsigned char* px, int* ex,
                           const int* sneed = nullptr, int qneed = 0) {
  __shared__ int s_e[RB];
  if (!mask[blockIdx.x]) return;
  // sneed (nullable): the planes only for matrices with sneed[b] > qneed (a
  // squaring that is not the matrix's last)
  if (sneed && sneed[blockIdx.x] <= qneed) px = nullptr;
  const BMat M = mats[blockIdx.x];
  const int n = M.d;
  const int r0 = blockIdx.y * RB;
  if (r0 >= n) return;
  const int nr = min(RB, n - r0);
  const int Mp = M.mtn * oz::TM, Np = M.ntn * oz::TN;
  const size_t pst = (size_t)Mp * Np;
  const long long* ab = acc + M.acc * 2;
  const T* Z1 = e.m1 ? (const T*)e.Z1 + M.off : nullptr;
  const T* Z2 = e.m2 ? (const T*)e.Z2 + M.off : nullptr;
  const int* fyb = fy + M.fo;
  T* Ob = out + M.off;
  // the weight combinations of this path's products
  const int key = e.gd ? -1 : e.am * 100 + e.m1 * 10 + e.m2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long bm = 0;
  for (int rr = w; rr < nr; rr += nw) {
    const int r = r0 + rr;
    const size_t ro = (size_t)r * n;
    const int er = exs[M.eo + r] - 64;
    const long long* a0 = ab + (size_t)r * Np * 2;
    const T* z1 = Z1 ? Z1 + ro : nullptr;
    const T* z2 = Z2 ? Z2 + ro : nullptr;
    T* o = Ob + ro;
    unsigned long long mx;
#define FM_EPI_ROW(AM, M1, M2) epi_row<T, AM, M1, M2>(e, a0, pst, er, fyb, z1, z2, o, n, r, lane)
    switch (key) {
      case 0: mx = FM_EPI_ROW(0, 0, 0); break;      // B^2
      case 12: mx = FM_EPI_ROW(0, 1, 2); break;     // residual C Y + C - Y
      case 112: mx = FM_EPI_ROW(1, 1, 2); break;    // residual u (B^2 Y) + C - Y
      case 11: mx = FM_EPI_ROW(0, 1, 1); break;     // correction Y + E + E Y
      case 13: mx = FM_EPI_ROW(0, 1, 3); break;     // F + G B + (sum a) B
      case 14: mx = FM_EPI_ROW(0, 1, 4); break;     // the same, complex sum
      case 30: mx = FM_EPI_ROW(0, 3, 0); break;     // squaring 2E + E E
      case 113: mx = FM_EPI_ROW(1, 1, 3); break;    // phi_1 doubling
      case 130: mx = FM_EPI_ROW(1, 3, 0); break;    // cos / sin doublings
      default: mx = FM_EPI_ROW(-1, -1, -1); break;
    }
#undef FM_EPI_ROW
    for (int o2 = 16; o2; o2 >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o2);
      mx = v > mx ? v : mx;
    }
    if (px && lane == 0) {
      s_e[rr] = oz::exp_above_bits(mx);
      ex[M.eo + r] = s_e[rr];
    }
    bm = mx > bm ? mx : bm;
  }
  if (emax && lane == 0 && bm) atomicMax(emax + blockIdx.x, bm);
  if (!px) return;
  __syncthreads();  // the block's rows of out_b and their exponents are in place
  row_planes<T>(M, Ob, r0, nr, s_e, px);
}

// One correction step's decision per matrix (the single-matrix rule):
// residual zero -> done; non-finite, too many steps or growing after 3 ->
// info -1, done; otherwise correct, and stop after that when em d <= 2^-30.
static __global__ void b_flags(int batch, const BMat* mats, const unsigned long long* emax, double* prev, int it,
                        int max_iters, int* mask_e, int* mask_u, int* info, int* active,
                        int* corrections, unsigned long long* emax_all) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  if (!mask_e[b]) {
    mask_u[b] = 0;
    return;
  }
  const double em = __longlong_as_double((long long)emax[b]);
  if (em == 0.0) {
    mask_e[b] = 0;
    mask_u[b] = 0;
  } else if (!(em < INFINITY) || it >= max_iters || (it >= 3 && em >= prev[b])) {
    if (info[b] == 0) info[b] = -1;
    mask_e[b] = 0;
    mask_u[b] = 0;
  } else {
    prev[b] = em;
    mask_u[b] = 1;
    atomicMax(corrections, it + 1);
    atomicMax(emax_all, emax[b]);
    if (em * mats[b].d <= 9.313225746154785e-10 /* 2^-30 */) mask_e[b] = 0;
  }
  if (mask_e[b]) atomicAdd(active, 1);
}

// W_b = V_b + Psi_b V_b (Phi = I + Psi), V_b, W_b d x m at voff: double
// products on the FP64 pipe (one product per call: O(d^2 m))
template <class T>
__global__ void b_apply(const BMat* mats, const int* mask, const T* Psi, const T* V, int m, T* W) {
  if (!mask[blockIdx.x]) return;
  const BMat M = mats[blockIdx.x];
  const int n = M.d;
  const int r0 = blockIdx.y * RB;
  if (r0 >= n) return;
  const int nr = min(RB, n - r0);
  const T* Pb = Psi + M.off;
  const T* Vb = V + M.voff;
  T* Wb = W + M.voff;
  for (int k = threadIdx.x; k < nr * m; k += blockDim.x) {
    const int r = r0 + k / m, c = k % m;
    T acc = Vb[(size_t)r * m + c];
    for (int q = 0; q < n; ++q) Tr<T>::mac(acc, Pb[(size_t)r * n + q], Vb[(size_t)q * m + c]);
    Wb[(size_t)r * m + c] = acc;
  }
}

// info[b] = code for every live matrix
static __global__ void b_set_info(int batch, const int* alive, int code, int* info) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch && alive[b]) info[b] = code;
}

// mask[b] = matrix b is alive and still has squaring q to do
static __global__ void b_square_mask(int batch, const int* alive, const int* s, int q, int* mask) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) mask[b] = alive[b] && q < s[b];
}

}  // namespace grid
}  // namespace fmk
