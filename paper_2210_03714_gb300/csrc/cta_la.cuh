// cta_la.cuh -- dense linear algebra executed by ONE thread block (CTA) on
// matrices that live in global memory (L2-resident working sets), with shared
// memory staging.  Used by the persistent kernels: each CTA owns one matrix
// of the batch at a time and runs every step of the method on it.
//
// Routines (all called by all NT threads of the CTA, with matching arguments):
//   cta_gemm     C = alpha A B + beta C        (64x64 tiles, 4x4 per thread)
//   cta_getrf    blocked right-looking LU with partial pivoting (LAPACK order:
//                piv[k] = row exchanged with row k at step k)
//   cta_getrs    solve (P^T L U) X = X, m right-hand sides, blocked
//   cta_getrs_t  solve (P^T L U)^T x = x, one right-hand side
// The factorization is the "LU decomposition and triangular solves" route the
// paper takes for each (I - c_i B)^{-1} (Sec. 1, first bullet of the dense case).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fmk {

constexpr int NT = 256;  // threads per CTA for every routine here

struct zd { double x, y; };
struct zf { float x, y; };

// ---------------------------------------------------------------------------
// scalar traits
// ---------------------------------------------------------------------------
template <class T> struct Tr;

template <> struct Tr<double> {
  using R = double;
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double one() { return 1.0; }
  static __device__ __forceinline__ double mag(double a) { return fabs(a); }
  static __device__ __forceinline__ void mac(double& c, double a, double b) { c = fma(a, b, c); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double rscale(double a, double s) { return __dmul_rn(a, s); }
  static __device__ __forceinline__ bool is_zero(double a) { return a == 0.0; }
  static __device__ __forceinline__ bool finite(double a) { return isfinite(a); }
};

template <> struct Tr<float> {
  using R = float;
  static __device__ __forceinline__ float zero() { return 0.0f; }
  static __device__ __forceinline__ float one() { return 1.0f; }
  static __device__ __forceinline__ float mag(float a) { return fabsf(a); }
  static __device__ __forceinline__ void mac(float& c, float a, float b) { c = fmaf(a, b, c); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return a / b; }
  static __device__ __forceinline__ float rscale(float a, float s) { return __fmul_rn(a, s); }
  static __device__ __forceinline__ bool is_zero(float a) { return a == 0.0f; }
  static __device__ __forceinline__ bool finite(float a) { return isfinite(a); }
};

template <> struct Tr<zd> {
  using R = double;
  static __device__ __forceinline__ zd zero() { return {0.0, 0.0}; }
  static __device__ __forceinline__ zd one() { return {1.0, 0.0}; }
  static __device__ __forceinline__ double mag(zd a) { return hypot(a.x, a.y); }
  static __device__ __forceinline__ void mac(zd& c, zd a, zd b) {
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
  }
  static __device__ __forceinline__ zd mul(zd a, zd b) {
    return {__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
            __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x))};
  }
  static __device__ __forceinline__ zd add(zd a, zd b) { return {__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)}; }
  static __device__ __forceinline__ zd sub(zd a, zd b) { return {__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)}; }
  static __device__ __forceinline__ zd div(zd a, zd b) {
    // scaled division (Smith): avoids overflow of |b|^2
    if (fabs(b.x) >= fabs(b.y)) {
      double r = b.y / b.x, den = b.x + b.y * r;
      return {(a.x + a.y * r) / den, (a.y - a.x * r) / den};
    } else {
      double r = b.x / b.y, den = b.x * r + b.y;
      return {(a.x * r + a.y) / den, (a.y * r - a.x) / den};
    }
  }
  static __device__ __forceinline__ zd rscale(zd a, double s) { return {__dmul_rn(a.x, s), __dmul_rn(a.y, s)}; }
  static __device__ __forceinline__ bool is_zero(zd a) { return a.x == 0.0 && a.y == 0.0; }
  static __device__ __forceinline__ bool finite(zd a) { return isfinite(a.x) && isfinite(a.y); }
};

template <> struct Tr<zf> {
  using R = float;
  static __device__ __forceinline__ zf zero() { return {0.0f, 0.0f}; }
  static __device__ __forceinline__ zf one() { return {1.0f, 0.0f}; }
  static __device__ __forceinline__ float mag(zf a) { return hypotf(a.x, a.y); }
  static __device__ __forceinline__ void mac(zf& c, zf a, zf b) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
  }
  static __device__ __forceinline__ zf mul(zf a, zf b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
  }
  static __device__ __forceinline__ zf add(zf a, zf b) { return {a.x + b.x, a.y + b.y}; }
  static __device__ __forceinline__ zf sub(zf a, zf b) { return {a.x - b.x, a.y - b.y}; }
  static __device__ __forceinline__ zf div(zf a, zf b) {
    if (fabsf(b.x) >= fabsf(b.y)) {
      float r = b.y / b.x, den = b.x + b.y * r;
      return {(a.x + a.y * r) / den, (a.y - a.x * r) / den};
    } else {
      float r = b.x / b.y, den = b.x * r + b.y;
      return {(a.x * r + a.y) / den, (a.y * r - a.x) / den};
    }
  }
  static __device__ __forceinline__ zf rscale(zf a, float s) { return {a.x * s, a.y * s}; }
  static __device__ __forceinline__ bool is_zero(zf a) { return a.x == 0.0f && a.y == 0.0f; }
  static __device__ __forceinline__ bool finite(zf a) { return isfinite(a.x) && isfinite(a.y); }
};

// conversions between the working (high) and factorization (low) types
template <class D, class S> __device__ __forceinline__ D cvt(S a);
template <> __device__ __forceinline__ double cvt<double, double>(double a) { return a; }
template <> __device__ __forceinline__ float cvt<float, double>(double a) { return __double2float_rn(a); }
template <> __device__ __forceinline__ double cvt<double, float>(float a) { return (double)a; }
template <> __device__ __forceinline__ float cvt<float, float>(float a) { return a; }
template <> __device__ __forceinline__ zd cvt<zd, zd>(zd a) { return a; }
template <> __device__ __forceinline__ zf cvt<zf, zd>(zd a) { return {__double2float_rn(a.x), __double2float_rn(a.y)}; }
template <> __device__ __forceinline__ zd cvt<zd, zf>(zf a) { return {(double)a.x, (double)a.y}; }
template <> __device__ __forceinline__ zf cvt<zf, zf>(zf a) { return a; }

// ---------------------------------------------------------------------------
// block reductions
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R cta_max(R v, R* red) {
  for (int o = 16; o; o >>= 1) {
    R w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (w > v || isnan(w)) ? w : v;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    R m = red[0];
    for (int w = 1; w < NT / 32; ++w) m = (red[w] > m || isnan(red[w])) ? red[w] : m;
    red[0] = m;
  }
  __syncthreads();
  R r = red[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int cta_or(int v, int* red) {
  v = __any_sync(0xffffffffu, v) ? 1 : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int r = 0;
  for (int w = 0; w < NT / 32; ++w) r |= red[w];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// GEMM: C[M x N] = alpha * A[M x K] * B[K x N] + beta * C  (row-major, ld*)
// beta == 0 means C is not read.  smem: 2 * 16 * 68 elements of T.
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 16, GLD = 68;

template <class T>
__device__ __noinline__ void cta_gemm(int M, int N, int K, typename Tr<T>::R alpha, const T* __restrict__ A,
                         int lda, const T* __restrict__ B, int ldb, typename Tr<T>::R beta,
                         T* C, int ldc, T* smem) {
  using TT = Tr<T>;
  T* sA = smem;             // [GK][GLD]  sA[k][m]
  T* sB = smem + GK * GLD;  // [GK][GLD]  sB[k][n]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int m0 = 0; m0 < M; m0 += GT)
    for (int n0 = 0; n0 < N; n0 += GT) {
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = TT::zero();
      // the next K chunk is loaded into registers while this one is used
      constexpr int PER = GT * GK / NT;
      T ra[PER], rb[PER];
      auto fetch = [&](int k0) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          int e = u * NT + tid;
          int r = e >> 4, kk = e & 15;
          int gr = m0 + r, gk = k0 + kk;
          ra[u] = (gr < M && gk < K) ? A[(size_t)gr * lda + gk] : TT::zero();
          int kb = e >> 6, c = e & 63;
          int gkb = k0 + kb, gc = n0 + c;
          rb[u] = (gkb < K && gc < N) ? B[(size_t)gkb * ldb + gc] : TT::zero();
        }
      };
      fetch(0);
      for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          int e = u * NT + tid;
          sA[(e & 15) * GLD + (e >> 4)] = ra[u];
          sB[(e >> 6) * GLD + (e & 63)] = rb[u];
        }
        __syncthreads();
        if (k0 + GK < K) fetch(k0 + GK);
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
          T a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = sA[kk * GLD + ty * 4 + i];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = sB[kk * GLD + tx * 4 + j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) TT::mac(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int r = m0 + ty * 4 + i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int c = n0 + tx * 4 + j;
          if (c >= N) continue;
          T v = TT::rscale(acc[i][j], alpha);
          if (beta != 0) v = TT::add(TT::rscale(C[(size_t)r * ldc + c], beta), v);
          C[(size_t)r * ldc + c] = v;
        }
      }
    }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// LU with partial pivoting, blocked right-looking, panel width NB.
// A: n x n (lda) in global memory, overwritten by L (unit, below) and U.
// piv: n ints (global).  Returns 0 or (first column with an exactly zero
// pivot) + 1.  smem: n*NB panel + GEMM tiles + reduction scratch.
// ---------------------------------------------------------------------------
template <class T, int NB>
__device__ __noinline__ int cta_getrf(int n, T* A, int lda, int* piv, T* smem) {
  using TT = Tr<T>;
  using R = typename TT::R;
  T* P = smem;                              // panel [n][NB]
  T* gsm = smem + (size_t)n * NB;           // GEMM tiles
  R* red = (R*)(gsm + 2 * GK * GLD);        // reduction scratch (8 R + 8 int)
  int* redi = (int*)(red + 8);
  __shared__ int s_piv, s_info, s_moved;
  __shared__ int s_pp[NB];
  const int tid = threadIdx.x;
  if (tid == 0) s_info = 0;
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int jb = min(NB, n - j0);
    const int rows = n - j0;
    // 1. load the panel
    for (int e = tid; e < rows * NB; e += NT) {
      int r = e / NB, c = e % NB;
      P[e] = (c < jb) ? A[(size_t)(j0 + r) * lda + j0 + c] : TT::zero();
    }
    __syncthreads();
    // 2. unblocked GEPP inside the panel
    for (int jj = 0; jj < jb; ++jj) {
      R best = -1;
      int bi = 0x7fffffff;
      for (int r = jj + tid; r < rows; r += NT) {
        R v = TT::mag(P[r * NB + jj]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o; o >>= 1) {
        R ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if ((tid & 31) == 0) { red[tid >> 5] = best; redi[tid >> 5] = bi; }
      __syncthreads();
      if (tid == 0) {
        R bb = red[0];
        int ii = redi[0];
        for (int w = 1; w < NT / 32; ++w)
          if (red[w] > bb || (red[w] == bb && redi[w] < ii)) { bb = red[w]; ii = redi[w]; }
        if (ii == 0x7fffffff) ii = jj;  // all NaN: keep the diagonal
        s_piv = ii;
        piv[j0 + jj] = j0 + ii;
        s_pp[jj] = j0 + ii;
        if (jj == 0) s_moved = 0;
        if (ii != jj) s_moved = 1;
      }
      __syncthreads();
      const int p = s_piv;
      if (p != jj && tid < NB) {
        T t = P[jj * NB + tid];
        P[jj * NB + tid] = P[p * NB + tid];
        P[p * NB + tid] = t;
      }
      __syncthreads();
      const T pv = P[jj * NB + jj];
      const bool zero = TT::is_zero(pv);
      if (zero && tid == 0 && s_info == 0) s_info = j0 + jj + 1;
      for (int r = jj + 1 + tid; r < rows; r += NT) {
        T l = P[r * NB + jj];
        if (!zero) l = TT::div(l, pv);
        P[r * NB + jj] = l;
        for (int c = jj + 1; c < jb; ++c) {
          T v = P[r * NB + c];
          T u = P[jj * NB + c];
          v = TT::sub(v, TT::mul(l, u));
          P[r * NB + c] = v;
        }
      }
      __syncthreads();
    }
    // 3. write the panel back
    for (int e = tid; e < rows * jb; e += NT) {
      int r = e / jb, c = e % jb;
      A[(size_t)(j0 + r) * lda + j0 + c] = P[r * NB + c];
    }
    // 4. apply the panel's row exchanges to the other columns (thread owns columns)
    for (int c = tid; c < n - jb && s_moved; c += NT) {
      int col = c < j0 ? c : c + jb;
      for (int jj = 0; jj < jb; ++jj) {
        int p = s_pp[jj];
        if (p != j0 + jj) {
          T t = A[(size_t)(j0 + jj) * lda + col];
          A[(size_t)(j0 + jj) * lda + col] = A[(size_t)p * lda + col];
          A[(size_t)p * lda + col] = t;
        }
      }
    }
    __syncthreads();
    // 5. U12 = L11^{-1} A12 (rows j0..j0+jb, columns j0+jb..n)
    for (int c = j0 + jb + tid; c < n; c += NT) {
      T x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) x[r] = (r < jb) ? A[(size_t)(j0 + r) * lda + c] : TT::zero();
#pragma unroll
      for (int r = 1; r < NB; ++r) {
#pragma unroll
        for (int l = 0; l < r; ++l) x[r] = TT::sub(x[r], TT::mul(P[r * NB + l], x[l]));
      }
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < jb) A[(size_t)(j0 + r) * lda + c] = x[r];
    }
    __syncthreads();
    // 6. trailing update A22 -= L21 U12
    if (j0 + jb < n)
      cta_gemm<T>(n - j0 - jb, n - j0 - jb, jb, (R)-1, A + (size_t)(j0 + jb) * lda + j0, lda,
                  A + (size_t)j0 * lda + j0 + jb, lda, (R)1, A + (size_t)(j0 + jb) * lda + j0 + jb,
                  lda, gsm);
    __syncthreads();
  }
  __syncthreads();
  int info = s_info;
  __syncthreads();
  return info;
}

// ---------------------------------------------------------------------------
// Solve (P^T L U) X = X for X: n x m (ldx), LU from cta_getrf.
// ---------------------------------------------------------------------------
template <class T, int NB>
__device__ __noinline__ void cta_getrs(int n, const T* LU, int lda, const int* piv, int m, T* X, int ldx,
                          T* smem) {
  using TT = Tr<T>;
  using R = typename TT::R;
  T* Lb = smem;                 // NB x NB diagonal block
  T* gsm = smem + NB * NB;      // GEMM tiles
  const int tid = threadIdx.x;
  // row exchanges, in order (thread owns columns)
  for (int c = tid; c < m; c += NT)
    for (int k = 0; k < n; ++k) {
      int p = piv[k];
      if (p != k) {
        T t = X[(size_t)k * ldx + c];
        X[(size_t)k * ldx + c] = X[(size_t)p * ldx + c];
        X[(size_t)p * ldx + c] = t;
      }
    }
  __syncthreads();
  // forward: unit lower
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int jb = min(NB, n - j0);
    for (int e = tid; e < NB * NB; e += NT) {
      int r = e / NB, c = e % NB;
      Lb[e] = (r < jb && c < jb) ? LU[(size_t)(j0 + r) * lda + j0 + c] : TT::zero();
    }
    __syncthreads();
    for (int c = tid; c < m; c += NT) {
      T x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) x[r] = (r < jb) ? X[(size_t)(j0 + r) * ldx + c] : TT::zero();
#pragma unroll
      for (int r = 1; r < NB; ++r) {
#pragma unroll
        for (int l = 0; l < r; ++l) x[r] = TT::sub(x[r], TT::mul(Lb[r * NB + l], x[l]));
      }
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < jb) X[(size_t)(j0 + r) * ldx + c] = x[r];
    }
    __syncthreads();
    if (j0 + jb < n)
      cta_gemm<T>(n - j0 - jb, m, jb, (R)-1, LU + (size_t)(j0 + jb) * lda + j0, lda,
                  X + (size_t)j0 * ldx, ldx, (R)1, X + (size_t)(j0 + jb) * ldx, ldx, gsm);
    __syncthreads();
  }
  // backward: upper
  for (int j0 = ((n - 1) / NB) * NB; j0 >= 0; j0 -= NB) {
    const int jb = min(NB, n - j0);
    for (int e = tid; e < NB * NB; e += NT) {
      int r = e / NB, c = e % NB;
      Lb[e] = (r < jb && c < jb) ? LU[(size_t)(j0 + r) * lda + j0 + c] : TT::one();
    }
    __syncthreads();
    for (int c = tid; c < m; c += NT) {
      T x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) x[r] = (r < jb) ? X[(size_t)(j0 + r) * ldx + c] : TT::zero();
#pragma unroll
      for (int r = NB - 1; r >= 0; --r) {
#pragma unroll
        for (int l = r + 1; l < NB; ++l) x[r] = TT::sub(x[r], TT::mul(Lb[r * NB + l], x[l]));
        x[r] = TT::div(x[r], Lb[r * NB + r]);
      }
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < jb) X[(size_t)(j0 + r) * ldx + c] = x[r];
    }
    __syncthreads();
    if (j0 > 0)
      cta_gemm<T>(j0, m, jb, (R)-1, LU + j0, lda, X + (size_t)j0 * ldx, ldx, (R)1, X, ldx, gsm);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Solve (P^T L U) X = X, with column slices of X resident in shared memory.
// For each slice of W columns: gather the rows through the pivot permutation,
// then forward and backward substitution by 16-row blocks, every update done
// in shared memory (the factors are read once per slice, 16-column panels
// staged in shared memory).  smem: n*W slice + 16*n panel + n ints.
// ---------------------------------------------------------------------------
template <class T>
__device__ __noinline__ void cta_getrs_sm(int n, const T* LU, int lda, const int* piv, int m,
                                          T* X, int ldx, T* smem, int W) {
  using TT = Tr<T>;
  constexpr int BK = 16;
  T* S = smem;                           // [n][W] slice
  T* Pn = smem + (size_t)n * W;          // [n][BK] panel (column block of L or U)
  int* perm = (int*)(Pn + (size_t)n * BK);
  const int tid = threadIdx.x;
  if (tid == 0) {  // compose the row exchanges into a gather permutation
    for (int k = 0; k < n; ++k) perm[k] = k;
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k) { int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
    }
  }
  __syncthreads();
  for (int c0 = 0; c0 < m; c0 += W) {
    const int w = min(W, m - c0);
    for (int e = tid; e < n * W; e += NT) {
      const int r = e / W, c = e % W;
      S[e] = c < w ? X[(size_t)perm[r] * ldx + c0 + c] : TT::zero();
    }
    __syncthreads();
    // forward, unit lower: block rows [j0, j0+jb)
    for (int j0 = 0; j0 < n; j0 += BK) {
      const int jb = min(BK, n - j0);
      // stage L[j0.., j0..j0+jb) (rows j0..n)
      for (int e = tid; e < (n - j0) * BK; e += NT) {
        const int r = e / BK, c = e % BK;
        Pn[e] = c < jb ? LU[(size_t)(j0 + r) * lda + j0 + c] : TT::zero();
      }
      __syncthreads();
      // diagonal block: one thread per column
      for (int c = tid; c < W; c += NT) {
        T x[BK];
#pragma unroll
        for (int r = 0; r < BK; ++r) x[r] = r < jb ? S[(size_t)(j0 + r) * W + c] : TT::zero();
#pragma unroll
        for (int r = 1; r < BK; ++r)
#pragma unroll
          for (int l = 0; l < r; ++l) x[r] = TT::sub(x[r], TT::mul(Pn[r * BK + l], x[l]));
#pragma unroll
        for (int r = 0; r < BK; ++r)
          if (r < jb) S[(size_t)(j0 + r) * W + c] = x[r];
      }
      __syncthreads();
      // rows below: S[r, :] -= L[r, j0:j0+jb] S[j0:j0+jb, :]
      for (int e = tid; e < (n - j0 - jb) * W; e += NT) {
        const int r = j0 + jb + e / W, c = e % W;
        T acc = S[(size_t)r * W + c];
        const T* Lr = Pn + (size_t)(r - j0) * BK;
#pragma unroll
        for (int l = 0; l < BK; ++l)
          if (l < jb) acc = TT::sub(acc, TT::mul(Lr[l], S[(size_t)(j0 + l) * W + c]));
        S[(size_t)r * W + c] = acc;
      }
      __syncthreads();
    }
    // backward, upper: block rows from the bottom
    for (int j0 = ((n - 1) / BK) * BK; j0 >= 0; j0 -= BK) {
      const int jb = min(BK, n - j0);
      // stage U[0..j0+jb, j0..j0+jb)
      for (int e = tid; e < (j0 + jb) * BK; e += NT) {
        const int r = e / BK, c = e % BK;
        Pn[e] = c < jb ? LU[(size_t)r * lda + j0 + c] : TT::zero();
      }
      __syncthreads();
      for (int c = tid; c < W; c += NT) {
        T x[BK];
#pragma unroll
        for (int r = 0; r < BK; ++r) x[r] = r < jb ? S[(size_t)(j0 + r) * W + c] : TT::zero();
#pragma unroll
        for (int r = BK - 1; r >= 0; --r) {
          if (r >= jb) continue;
#pragma unroll
          for (int l = r + 1; l < BK; ++l)
            if (l < jb) x[r] = TT::sub(x[r], TT::mul(Pn[(j0 + r) * BK + l], x[l]));
          x[r] = TT::div(x[r], Pn[(j0 + r) * BK + r]);
        }
#pragma unroll
        for (int r = 0; r < BK; ++r)
          if (r < jb) S[(size_t)(j0 + r) * W + c] = x[r];
      }
      __syncthreads();
      for (int e = tid; e < j0 * W; e += NT) {
        const int r = e / W, c = e % W;
        T acc = S[(size_t)r * W + c];
        const T* Ur = Pn + (size_t)r * BK;
#pragma unroll
        for (int l = 0; l < BK; ++l)
          if (l < jb) acc = TT::sub(acc, TT::mul(Ur[l], S[(size_t)(j0 + l) * W + c]));
        S[(size_t)r * W + c] = acc;
      }
      __syncthreads();
    }
    for (int e = tid; e < n * W; e += NT) {
      const int r = e / W, c = e % W;
      if (c < w) X[(size_t)r * ldx + c0 + c] = S[e];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Solve (P^T L U) X = X, left-looking by 16-row blocks.  Block j of the
// solution is X_j = D_j^{-1} (X_j - F_j X_known) with F_j the already solved
// part of row block j of L (forward) or U (backward), staged k-major in shared
// memory.  Each thread owns one column (and a share of k when m < NT) and
// keeps the 16 rows of its column block in registers: per k one global load
// of X, four broadcast shared loads and 16 FMAs; every block of X is written
// once.  smem: 16*n panel + NT*16 partial sums.
// ---------------------------------------------------------------------------
template <class T>
__device__ __noinline__ void cta_getrs_ll(int n, const T* LU, int lda, const int* piv, int m,
                                          T* X, int ldx, T* smem) {
  using TT = Tr<T>;
  constexpr int BK = 16;
  T* Pn = smem;                       // [k][BK]
  T* part = smem + (size_t)BK * n;    // [group][BK][lane-column]
  const int tid = threadIdx.x;
  const int G = m >= NT ? 1 : min(BK, NT / m);  // groups sharing the k loop
  const int cpp = NT / G;                       // columns per pass
  const int g = tid / cpp, cl = tid % cpp;
  // when G does not divide NT, the last NT - G cpp threads have no group: they
  // only take part in the barriers
  const bool busy = g < G;
  // row exchanges, in order (thread owns columns); none when piv is the identity
  int moved = 0;
  for (int k = tid; k < n; k += NT) moved |= (piv[k] != k);
  if (__syncthreads_or(moved))
    for (int c = tid; c < m; c += NT)
      for (int k = 0; k < n; ++k) {
        const int p = piv[k];
        if (p != k) {
          T t = X[(size_t)k * ldx + c];
          X[(size_t)k * ldx + c] = X[(size_t)p * ldx + c];
          X[(size_t)p * ldx + c] = t;
        }
      }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {  // 0: forward with L, 1: backward with U
    const int nblk = (n + BK - 1) / BK;
    for (int bi = 0; bi < nblk; ++bi) {
      const int j0 = pass == 0 ? bi * BK : (nblk - 1 - bi) * BK;
      const int jb = min(BK, n - j0);
      // known range of k and the staged panel Pn[k][r] = F(j0 + r, k)
      const int k0 = pass == 0 ? 0 : j0 + jb, k1 = pass == 0 ? j0 : n;
      // rows j0..j0+jb of the factor, read along the row (coalesced), stored
      // k-major: the known part [k0, k1), then the diagonal block [j0, j0+jb)
      {
        const int nk = k1 - k0 + jb;
        for (int e = tid; e < nk * BK; e += NT) {
          const int r = e / nk, kk = e % nk;
          const int k = kk < k1 - k0 ? k0 + kk : j0 + (kk - (k1 - k0));
          Pn[kk * BK + r] = r < jb ? LU[(size_t)(j0 + r) * lda + k] : TT::zero();
        }
      }
      __syncthreads();
      for (int c0 = 0; c0 < m; c0 += cpp) {
        const int c = c0 + cl;
        T acc[BK];
#pragma unroll
        for (int r = 0; r < BK; ++r) acc[r] = TT::zero();
        if (busy && c < m) {
          const int kn = k1 - k0;
          const int kb = (kn * g) / G, ke = (kn * (g + 1)) / G;
          // eight loads in flight per thread before their FMAs
          int kk = kb;
          for (; kk + 8 <= ke; kk += 8) {
            T x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = X[(size_t)(k0 + kk + u) * ldx + c];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const T* pr = Pn + (size_t)(kk + u) * BK;
#pragma unroll
              for (int r = 0; r < BK; ++r) TT::mac(acc[r], pr[r], x[u]);
            }
          }
          for (; kk < ke; ++kk) {
            const T x = X[(size_t)(k0 + kk) * ldx + c];
            const T* pr = Pn + (size_t)kk * BK;
#pragma unroll
            for (int r = 0; r < BK; ++r) TT::mac(acc[r], pr[r], x);
          }
        }
        if (G > 1) {
          if (busy)
#pragma unroll
            for (int r = 0; r < BK; ++r) part[((size_t)g * BK + r) * cpp + cl] = acc[r];
          __syncthreads();
          if (g == 0)
            for (int h = 1; h < G; ++h)
#pragma unroll
              for (int r = 0; r < BK; ++r)
                acc[r] = TT::add(acc[r], part[((size_t)h * BK + r) * cpp + cl]);
        }
        if (g == 0 && c < m) {
          T x[BK];
#pragma unroll
          for (int r = 0; r < BK; ++r)
            x[r] = r < jb ? TT::sub(X[(size_t)(j0 + r) * ldx + c], acc[r]) : TT::zero();
          const T* D = Pn + (size_t)(k1 - k0) * BK;  // D[l][r] = F(j0 + r, j0 + l)
          if (pass == 0) {
#pragma unroll
            for (int r = 1; r < BK; ++r)
#pragma unroll
              for (int l = 0; l < r; ++l) x[r] = TT::sub(x[r], TT::mul(D[l * BK + r], x[l]));
          } else {
#pragma unroll
            for (int r = BK - 1; r >= 0; --r) {
              if (r >= jb) continue;
#pragma unroll
              for (int l = r + 1; l < BK; ++l)
                if (l < jb) x[r] = TT::sub(x[r], TT::mul(D[l * BK + r], x[l]));
              x[r] = TT::div(x[r], D[r * BK + r]);
            }
          }
#pragma unroll
          for (int r = 0; r < BK; ++r)
            if (r < jb) X[(size_t)(j0 + r) * ldx + c] = x[r];
        }
        if (G > 1) __syncthreads();
      }
      __syncthreads();
    }
  }
}

// slice width that fits the shared memory budget (elements of T)
__host__ __device__ inline int getrs_width(int n, int m, size_t budget_elems) {
  long w = (long)((budget_elems - 16L * n - n) / n);
  if (w > 64) w = 64;
  if (w > m) w = m;
  if (w < 1) w = 1;
  return (int)w;
}

}  // namespace fmk
