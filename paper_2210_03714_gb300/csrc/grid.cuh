// grid.cuh -- kernels of the grid-wide path: one matrix of large order d
// spread over every SM (the one-CTA-per-matrix kernels stop at d = 1024).
//
// Every step of the method is a matrix product or an elementwise pass:
//   a1/a2   column sums of |tA| (eta), B = tA / 2^s or (t/N) A      -> colsum, scale
//   a3-a5   each shifted system (I - c_i B) Y_i = c_i B is solved by the
//           residual-correction iteration Y <- Y + (I + Y) E with
//           E = C - (I - C) Y, C = c_i B (Newton-Schulz for the inverse, kept
//           in the deviation Y = (I - C)^{-1} - I, which equals the roundoff-
//           form term Y_i of Eq. ParallRoundOff)                 -> products
//   a6      F = a0 I + d1 B + d2 B^2 + sum_i b_i Y_i              -> axpy
//   a7      squarings E <- 2E + E E (F = I + E), phi_1 doublings, or N steps
//           W <- W + E W for the action                          -> products
// Products run either on the tensor cores (digit planes, exact FP32
// accumulation, integer partial sums added atomically across K-splits) or on
// the FP64 pipe (64 x 64 CTA tiles); the same epilogue kernel then forms
// out = alpha P + beta1 Z1 + beta2 Z2 + gamma I.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cta_la.cuh"
#include "ozaki.cuh"
#include "tc.cuh"

namespace fmk {
namespace grid {

// ---- element access for real (double) and complex (zd) matrices ------------
template <class T> struct El;
template <> struct El<double> {
  static constexpr int parts = 1;
  static __device__ __forceinline__ double re(double a) { return a; }
  static __device__ __forceinline__ double im(double) { return 0.0; }
  static __device__ __forceinline__ double make(double r, double) { return r; }
};
template <> struct El<zd> {
  static constexpr int parts = 2;
  static __device__ __forceinline__ double re(zd a) { return a.x; }
  static __device__ __forceinline__ double im(zd a) { return a.y; }
  static __device__ __forceinline__ zd make(double r, double i) { return {r, i}; }
};

// largest |re|, |im| as the bit pattern of a non-negative double (integer ops)
template <class T>
__device__ __forceinline__ unsigned long long abs_bits(T v);

// (cr + i ci) * a with one rounding per real operation (real: cr * a)
template <class T> __device__ __forceinline__ T cmul(double cr, double ci, T a);
template <> __device__ __forceinline__ double cmul<double>(double cr, double, double a) {
  return __dmul_rn(cr, a);
}
template <> __device__ __forceinline__ zd cmul<zd>(double cr, double ci, zd a) {
  return Tr<zd>::mul(zd{cr, ci}, a);
}

// a + (cr + i ci) z: an add or a subtract when the coefficient is +-1
template <class T>
__device__ __forceinline__ T axpy1(T a, double cr, double ci, T z) {
  if (ci == 0 && cr == 1.0) return Tr<T>::add(a, z);
  if (ci == 0 && cr == -1.0) return Tr<T>::sub(a, z);
  return Tr<T>::add(a, cmul<T>(cr, ci, z));
}

template <>
__device__ __forceinline__ unsigned long long abs_bits<double>(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
}
template <>
__device__ __forceinline__ unsigned long long abs_bits<zd>(zd v) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFULL;
  const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFULL;
  return a > b ? a : b;
}


// ---- a1: finiteness of A, B = t A (one rounding), column sums of |B| -------
// One thread per column; rows in ascending order (the order of the one-CTA
// kernels, so both paths pick the same s).
template <class T>
__global__ void colsum_scale(int n, const T* A, int lda, double t, T* B, double* colsum,
                             int* nonfinite) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double s = 0;
  int bad = 0;
  for (int r = 0; r < n; ++r) {
    const T a = A[(size_t)r * lda + c];
    bad |= !Tr<T>::finite(a);
    const T b = Tr<T>::rscale(a, t);
    B[(size_t)r * n + c] = b;
    s += Tr<T>::mag(b);
  }
  colsum[c] = s;
  if (bad) atomicOr(nonfinite, 1);
}

// eta = max column sum (NaN propagates, as in the one-CTA kernels)
static __global__ void colsum_max(int n, const double* colsum, double* eta) {
  __shared__ double red[32];
  double m = 0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const double s = colsum[c];
    m = (s > m || isnan(s)) ? s : m;
  }
  for (int o = 16; o; o >>= 1) {
    const double v = __shfl_xor_sync(0xffffffffu, m, o);
    m = (v > m || isnan(v)) ? v : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) r = (red[w] > r || isnan(red[w])) ? red[w] : r;
    *eta = r;
  }
}

// B = ldexp(B, -s) in place (exact)
template <class T>
__global__ void pow2_scale(size_t count, T* B, int s) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    T b = B[e];
    B[e] = El<T>::make(ldexp(El<T>::re(b), -s), ldexp(El<T>::im(b), -s));
  }
}

// B = h A (action: one rounding, as the one-CTA kernels)
template <class T>
__global__ void scale_into(int n, const T* A, int lda, double h, T* B) {
  const size_t count = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    B[e] = Tr<T>::rscale(A[(size_t)r * lda + c], h);
  }
}

// C = c B (one rounding per real operation); Y = C (first iterate: (I - C)^-1 ~ I + C)
template <class T>
__global__ void build_shift(size_t count, const T* B, double cr, double ci, T* C, T* Y) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const T v = cmul<T>(cr, ci, B[e]);
    C[e] = v;
    Y[e] = v;
  }
}

// C = u1 B + u2 B2 (each product rounded once; C = u2 B2 when u1 = 0); Y = C
template <class T>
__global__ void build_shift2(size_t count, const T* B, double u1r, double u1i, const T* B2,
                             double u2r, double u2i, T* C, T* Y) {
  const bool one = u1r == 0.0 && u1i == 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    T v = cmul<T>(u2r, u2i, B2[e]);
    if (!one) v = Tr<T>::add(cmul<T>(u1r, u1i, B[e]), v);
    C[e] = v;
    Y[e] = v;
  }
}

// The first correction step of a system C = u B^2 (u real) from powers of B
// shared by every such system: from Y = C the residual is u^2 B^4 and the
// update E Y + Y + E is u^3 B^6 + u B^2 + u^2 B^4 (in the update's order of
// additions).  C = u B^2 and Y = that first iterate.
template <class T>
__global__ void pair_first(size_t count, double u, double u2, double u3, const T* B2, const T* B4,
                           const T* B6, T* C, T* Y) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const T c = Tr<T>::rscale(B2[e], u);
    const T p = Tr<T>::rscale(B6[e], u3);
    C[e] = c;
    Y[e] = Tr<T>::add(Tr<T>::add(p, c), Tr<T>::rscale(B4[e], u2));
  }
}

// a fused +-c pair with Y = (I - c^2 B^2)^-1 - I: F += s Y and G += a Y
// (G = a Y for the first pair), s = b+ + b-, a = (b+ - b-) c
template <class T>
__global__ void pair_acc(size_t count, double sr, double si, double ar, double ai, const T* Y,
                         int first, T* F, T* G) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const T y = Y[e];
    F[e] = Tr<T>::add(F[e], cmul<T>(sr, si, y));
    const T g = cmul<T>(ar, ai, y);
    G[e] = first ? g : Tr<T>::add(G[e], g);
  }
}

// F (n x n, ld n) = base I + d1 B + d2 B2   (B2 nullable when d2 == 0)
template <class T>
__global__ void init_f(int n, double base, double d1, const T* B, double d2, const T* B2, T* F) {
  const size_t count = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    T v = Tr<T>::rscale(r == c ? Tr<T>::one() : Tr<T>::zero(), base);
    if (d1 != 0) v = Tr<T>::add(v, Tr<T>::rscale(B[e], d1));
    if (d2 != 0) v = Tr<T>::add(v, Tr<T>::rscale(B2[e], d2));
    F[e] = v;
  }
}

// F += b Y  (roundoff form) or F += b (I + Y) (plain form)
template <class T>
__global__ void accumulate(int n, double br, double bi, const T* Y, int plain, T* F) {
  const size_t count = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    T y = Y[e];
    if (plain && r == c) y = Tr<T>::add(y, Tr<T>::one());
    F[e] = Tr<T>::add(F[e], cmul<T>(br, bi, y));
  }
}

// out (rows x cols, ldo) = in (ld ldi) + g I
template <class T>
__global__ void add_identity(int rows, int cols, const T* in, int ldi, double g, T* out, int ldo) {
  const size_t count = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e % cols);
    T v = in[(size_t)r * ldi + c];
    if (r == c) v = Tr<T>::add(v, Tr<T>::rscale(Tr<T>::one(), g));
    out[(size_t)r * ldo + c] = v;
  }
}

// copy with leading dimensions, and a finiteness check of the source
template <class T>
__global__ void copy_check(int rows, int cols, const T* in, int ldi, T* out, int ldo,
                           int* nonfinite) {
  const size_t count = (size_t)rows * cols;
  int bad = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e % cols);
    const T v = in[(size_t)r * ldi + c];
    bad |= !Tr<T>::finite(v);
    out[(size_t)r * ldo + c] = v;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(nonfinite, 1);
}

// ---- products: epilogue --------------------------------------------------
// out[i][j] = alpha P_ij + b1 Z1_ij + b2 Z2_ij + (i == j ? g : 0), complex
// coefficients (real matrices use the real parts).  P comes from the exact
// integer sums of the tensor-core product (acc != nullptr) or from a double
// matrix Pd.  out may alias Z1 or Z2 (same element read, then written).
struct Epi {
  double ar = 1, ai = 0;
  const void* Z1 = nullptr;
  int ld1 = 0;
  double b1r = 0, b1i = 0;
  const void* Z2 = nullptr;
  int ld2 = 0;
  double b2r = 0, b2i = 0;
  double gr = 0, gi = 0;
  unsigned long long* maxabs = nullptr;  // max |re|, |im| of out (bits), nullable
  // integer form (fx = 1, set by fixed_form): alpha, b1, b2 are real powers of
  // two (sign s*, exponent k*), and each output is summed exactly in 128-bit
  // fixed point and rounded once, without the FP64 unit
  int fx = 0, ka = 0, sa = 0, k1 = 0, s1 = 0, k2 = 0, s2 = 0;
  // light form (fx = 2): alpha = 1 and b1, b2 = +-1 (or absent); P is rounded
  // once and Z1, Z2 added with two double operations (m*: 1 add, 2 subtract)
  int m1 = 0, m2 = 0;
};

// c = +-2^k
inline bool epi_pow2(double c, int* neg, int* k) {
  if (!(c != 0) || !(c - c == 0)) return false;
  int e;
  const double m = frexp(c < 0 ? -c : c, &e);
  if (m != 0.5) return false;
  *neg = c < 0;
  *k = e - 1;
  return true;
}

// select the light form, else the integer form, when the coefficients allow (host)
inline void fixed_form(Epi& e) {
  e.fx = 0;
  if (e.ai != 0 || e.b1i != 0 || e.b2i != 0) return;
  auto pm1 = [](const void* z, double b) { return !z ? 0 : (b == 1.0 ? 1 : (b == -1.0 ? 2 : -1)); };
  e.m1 = pm1(e.Z1, e.b1r);
  e.m2 = pm1(e.Z2, e.b2r);
  if (e.ar == 1.0 && e.m1 >= 0 && e.m2 >= 0) {
    e.fx = 2;
    return;
  }
  if (!epi_pow2(e.ar, &e.sa, &e.ka) || e.ka < -2) return;
  if (e.Z1 && !epi_pow2(e.b1r, &e.s1, &e.k1)) return;
  if (e.Z2 && !epi_pow2(e.b2r, &e.s2, &e.k2)) return;
  e.fx = 1;
}

// one component of alpha P + b1 z1 + b2 z2 + g, P = (hi 2^24 + lo) 2^e2: exact
// 128-bit sum rounded once (integer form), else in double
__device__ __forceinline__ double epi_part(const Epi& e, long long hi, long long lo, int e2,
                                           bool h1, double z1, bool h2, double z2, bool diag,
                                           double g) {
  if (e.fx == 2) {
    double v = oz::combine_scaled(hi, lo, e2);
    if (e.m1) v = e.m1 == 1 ? __dadd_rn(v, z1) : __dsub_rn(v, z1);
    if (e.m2) v = e.m2 == 1 ? __dadd_rn(v, z2) : __dsub_rn(v, z2);
    if (diag && g != 0) v = __dadd_rn(v, g);
    return v;
  }
  if (e.fx == 1) {
    const int u = e2 - 2;  // two fraction bits below the product's unit (alpha >= 1/4)
    __int128 S = (((__int128)hi << 24) + (__int128)lo) << 2;
    S = e.ka >= 0 ? (S << e.ka) : (S >> (-e.ka));
    if (e.sa) S = -S;
    bool ok = true;
    __int128 t;
    if (h1) {
      ok &= oz::to_fixed(z1, e.k1, e.s1, u, t);
      S += t;
    }
    if (h2) {
      ok &= oz::to_fixed(z2, e.k2, e.s2, u, t);
      S += t;
    }
    if (diag && g != 0) {
      ok &= oz::to_fixed(g, 0, false, u, t);
      S += t;
    }
    if (ok) return oz::round_i128(S, u);
  }
  // a term too far above the product's scale, not finite, or general weights
  double v = oz::combine_scaled(hi, lo, e2);
  if (e.ar != 1.0) v = __dmul_rn(e.ar, v);
  if (h1) v = __dadd_rn(v, __dmul_rn(e.b1r, z1));
  if (h2) v = __dadd_rn(v, __dmul_rn(e.b2r, z2));
  if (diag && g != 0) v = __dadd_rn(v, g);
  return v;
}

template <class T>
__global__ void epilogue(int M, int N, const long long* acc, int parts, int Mp, int Np,
                         const int* ex, const int* fy, const T* Pd, int ldp, Epi e, T* out,
                         int ldo) {
  const size_t count = (size_t)M * N;
  unsigned long long mx = 0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count;
       k += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(k / N), j = (int)(k % N);
    T v;
    if (acc && e.fx) {
      const int e2 = ex[i] + fy[j] - 64;
      const long long* a0 = acc + ((size_t)i * Np + j) * 2;
      const T z1 = e.Z1 ? ((const T*)e.Z1)[(size_t)i * e.ld1 + j] : El<T>::make(0.0, 0.0);
      const T z2 = e.Z2 ? ((const T*)e.Z2)[(size_t)i * e.ld2 + j] : El<T>::make(0.0, 0.0);
      const double re = epi_part(e, a0[0], a0[1], e2, e.Z1, El<T>::re(z1), e.Z2, El<T>::re(z2),
                                 i == j, e.gr);
      double im = 0;
      if (parts == 2) {
        const long long* a1 = acc + ((size_t)Mp * Np + (size_t)i * Np + j) * 2;
        im = epi_part(e, a1[0], a1[1], e2, e.Z1, El<T>::im(z1), e.Z2, El<T>::im(z2), i == j,
                      e.gi);
      }
      v = El<T>::make(re, im);
    } else {
      double pr, pi = 0;
      if (acc) {
        const int e2 = ex[i] + fy[j] - 64;
        const long long* a0 = acc + ((size_t)i * Np + j) * 2;
        pr = oz::combine_scaled(a0[0], a0[1], e2);
        if (parts == 2) {
          const long long* a1 = acc + ((size_t)Mp * Np + (size_t)i * Np + j) * 2;
          pi = oz::combine_scaled(a1[0], a1[1], e2);
        }
      } else {
        const T p = Pd[(size_t)i * ldp + j];
        pr = El<T>::re(p);
        pi = El<T>::im(p);
      }
      v = El<T>::make(pr, pi);
      if (e.ar != 1.0 || e.ai != 0) v = cmul<T>(e.ar, e.ai, v);
      if (e.Z1) v = axpy1<T>(v, e.b1r, e.b1i, ((const T*)e.Z1)[(size_t)i * e.ld1 + j]);
      if (e.Z2) v = axpy1<T>(v, e.b2r, e.b2i, ((const T*)e.Z2)[(size_t)i * e.ld2 + j]);
      if (i == j && (e.gr != 0 || e.gi != 0)) v = Tr<T>::add(v, El<T>::make(e.gr, e.gi));
    }
    out[(size_t)i * ldo + j] = v;
    const unsigned long long ab = abs_bits<T>(v);
    mx = ab > mx ? ab : mx;
  }
  if (e.maxabs) {
    for (int o = 16; o; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = v > mx ? v : mx;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(e.maxabs, mx);
  }
}

// ---- products on the FP64 pipe: one 64 x 64 output tile per CTA ------------
template <class T>
__global__ void __launch_bounds__(NT, 2) dgemm_tiles(int M, int N, int K, const T* X, int ldx,
                                                     const T* Y, int ldy, T* P, int ldp) {
  __shared__ __align__(16) T sm[2 * GK * GLD];
  const int ntn = (N + GT - 1) / GT;
  const int mt = blockIdx.x / ntn, nt = blockIdx.x % ntn;
  const int m0 = mt * GT, n0 = nt * GT;
  cta_gemm<T>(min(GT, M - m0), min(GT, N - n0), K, 1.0, X + (size_t)m0 * ldx, ldx, Y + n0, ldy,
              0.0, P + (size_t)m0 * ldp + n0, ldp, sm);
}

// ---- products on the tensor cores ------------------------------------------
// Digit planes in global memory: for plane set s, row tile mt (128 rows) and
// K chunk c (16 values), GXST bytes at  px + s * pxs + (mt * kc + c) * GXST
// (7 planes of 128 x 16 BF16 in 8 x 16-byte core matrices, K-major), likewise
// Y with column tiles of 64 (GYST bytes).  A complex operand has sets (re, im)
// for X and (re, im, -im) for Y, all sharing one exponent per row (column).
constexpr int GKC = 16;                          // K per stage: one MMA K-step
constexpr int GSTEPS = 7;                        // stages per exact group: K = 112
constexpr int GNST = 4;                          // stages in the ring
constexpr int GNACC = 7;                         // accumulators: levels 2..8
constexpr uint32_t GXB = oz::TM * GKC * 2;       // one X plane of a stage (4 KB)
constexpr uint32_t GYB = oz::TN * GKC * 2;       // one Y plane (2 KB)
constexpr uint32_t GXST = oz::S * GXB;           // 28672
constexpr uint32_t GYST = oz::S * GYB;           // 14336
constexpr uint32_t GST = GXST + GYST;            // 43008
constexpr uint32_t GSMEM = GNST * GST;           // 172032
constexpr int GRW = 16;                          // readout warps: 4 per TMEM lane quarter
constexpr int GTHREADS = GRW * 32 + 32;          // readout warps + 1 producer / MMA warp

__device__ __forceinline__ uint32_t plane_off16(int r, int k) {
  return (uint32_t)(((r >> 3) * (GKC / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// largest |re|, |im| of every row of X (bits, dst zeroed by the caller)
template <class T>
__global__ void row_max(int M, int K, const T* X, int ldx, unsigned long long* rmax) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = w; r < M; r += nw) {
    unsigned long long mx = 0;  // as bits: integer operations only
    for (int k = lane; k < K; k += 32) {
      const unsigned long long b = abs_bits<T>(X[(size_t)r * ldx + k]);
      mx = b > mx ? b : mx;
    }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = b > mx ? b : mx;
    }
    if (lane == 0) rmax[r] = mx;
  }
}

// largest |re|, |im| of every column of Y: blocks of 32 columns x 8 row lanes
template <class T>
__global__ void col_max(int K, int N, const T* Y, int ldy, unsigned long long* cmax) {
  __shared__ unsigned long long red[8][33];
  const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + cx;
  unsigned long long mx = 0;
  if (j < N)
    for (int k = blockIdx.y * 8 + ry; k < K; k += 8 * gridDim.y) {
      const unsigned long long b = abs_bits<T>(Y[(size_t)k * ldy + j]);
      mx = b > mx ? b : mx;
    }
  red[ry][cx] = mx;
  __syncthreads();
  if (ry == 0 && j < N) {
    for (int q = 1; q < 8; ++q) mx = red[q][cx] > mx ? red[q][cx] : mx;
    atomicMax(cmax + j, mx);
  }
}

__device__ __forceinline__ int exp_of_bits(unsigned long long b) { return oz::exp_above_bits(b); }

// X (M x K) -> row digit planes; item = (row, 8 consecutive k)
template <class T>
__global__ void split_rows(int M, int K, const T* X, int ldx, const unsigned long long* rmax,
                           unsigned char* px, size_t pxs, int kc, int* ex) {
  const int mtn = (M + oz::TM - 1) / oz::TM;
  const long long items = (long long)mtn * oz::TM * kc * (GKC / 8);
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int k8 = (int)(it % (kc * (GKC / 8)));
    const int r = (int)(it / (kc * (GKC / 8)));
    const int e = r < M ? exp_of_bits(rmax[r]) : 0;
    if (k8 == 0) ex[r] = e;
    __align__(16) __nv_bfloat16 dr[oz::S][8], di[oz::S][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k8 * 8 + j;
      const T v = (r < M && k < K) ? X[(size_t)r * ldx + k] : El<T>::make(0.0, 0.0);
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
    const int tile = r / oz::TM, chunk = (k8 * 8) / GKC;
    const size_t blk = ((size_t)tile * kc + chunk) * GXST;
    const uint32_t off = plane_off16(r % oz::TM, (k8 * 8) % GKC);
#pragma unroll
    for (int p = 0; p < oz::S; ++p) *(uint4*)(px + blk + p * GXB + off) = *(const uint4*)dr[p];
    if (El<T>::parts == 2) {
#pragma unroll
      for (int p = 0; p < oz::S; ++p)
        *(uint4*)(px + pxs + blk + p * GXB + off) = *(const uint4*)di[p];
    }
  }
}

// Y (K x N) -> column digit planes (N-major); item = (column, 8 consecutive k)
template <class T>
__global__ void split_cols(int K, int N, const T* Y, int ldy, const unsigned long long* cmax,
                           unsigned char* py, size_t pys, int kc, int* fy) {
  const int ntn = (N + oz::TN - 1) / oz::TN;
  const long long items = (long long)ntn * oz::TN * kc * (GKC / 8);
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(it % (ntn * oz::TN));
    const int k8 = (int)(it / (ntn * oz::TN));
    const int e = j < N ? exp_of_bits(cmax[j]) : 0;
    if (k8 == 0) fy[j] = e;
    __align__(16) __nv_bfloat16 dr[oz::S][8], di[oz::S][8], dn[oz::S][8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int k = k8 * 8 + jj;
      const T v = (j < N && k < K) ? Y[(size_t)k * ldy + j] : El<T>::make(0.0, 0.0);
      __nv_bfloat16 t[oz::S];
      oz::digits(El<T>::re(v), e, t);
#pragma unroll
      for (int p = 0; p < oz::S; ++p) dr[p][jj] = t[p];
      if (El<T>::parts == 2) {
        oz::digits(El<T>::im(v), e, t);
#pragma unroll
        for (int p = 0; p < oz::S; ++p) {
          di[p][jj] = t[p];
          dn[p][jj] = __hneg(t[p]);
        }
      }
    }
    const int tile = j / oz::TN, chunk = (k8 * 8) / GKC;
    const size_t blk = ((size_t)tile * kc + chunk) * GYST;
    const uint32_t off = plane_off16(j % oz::TN, (k8 * 8) % GKC);
#pragma unroll
    for (int p = 0; p < oz::S; ++p) *(uint4*)(py + blk + p * GYB + off) = *(const uint4*)dr[p];
    if (El<T>::parts == 2) {
#pragma unroll
      for (int p = 0; p < oz::S; ++p) {
        *(uint4*)(py + pys + blk + p * GYB + off) = *(const uint4*)di[p];
        *(uint4*)(py + 2 * pys + blk + p * GYB + off) = *(const uint4*)dn[p];
      }
    }
  }
}

// Work item: output tile (mt, nt) of part `part` over a range of exact
// groups (112 values of the concatenated K).  The part's K runs over nseg
// segments, segment g pairing X plane set sx[part][g] with Y plane set
// sy[part][g] (complex: re = Xr Yr + Xi (-Yi), im = Xr Yi + Xi Yr).  The
// kernel is persistent: each CTA takes items blockIdx.x, + gridDim.x, ...
//
// Accumulator a (TMEM columns 64a .. 64a + 63) holds level L = a + 2 (digit
// pairs p + q = L).  Bounds at K = 112 in units of the level (|d_1| <= 256,
// |d_p| <= 128 for p > 1): L = 2: 2^23, 3: 2^23, 4: 1.25 2^23, 5: 1.5 2^23,
// 6: 1.75 2^23, 7: 1.75 2^23, 8: 1.97 2^23 -- every partial sum is an integer
// below 2^24 units, exact in FP32 whatever the adder's rounding.  For digit p
// of X, the Y planes q = 1 .. 8 - p are adjacent in shared memory and their
// accumulators adjacent in TMEM, so one MMA of N = 64 (8 - p) (split at 256)
// covers them: 10 MMAs per K step.
//
// Warps 0-15 read the accumulators after each group (warp w: TMEM lanes
// 32 (w % 4) .. + 31, columns 16 (w / 4) .. + 15 of every accumulator) into
// two exact 64-bit sums per output; warp 16 lane 0 keeps a ring of 4 stages
// filled by bulk copies and issues the MMAs.  mbarriers: full[s] (copies
// landed), empty[s] (the stage's MMAs finished), accf (a group's MMAs
// finished), accr (the 16 readout warps released the accumulators).
// One matrix of a batch on the tensor-core product path: its geometry and
// where its data sits in the batch-wide buffers.
struct BMat {
  int d, mtn, ntn, kc;  // order, 128-row tiles, 64-column tiles, 16-value K chunks
  long long off;        // element offset in the packed work matrices (leading dimension d)
  long long uoff;       // element offset of the caller's matrix (A in, F out)
  long long px, py;     // byte offsets of its X and Y digit planes
  long long acc;        // offset, in (hi, lo) pairs, of its accumulators
  int eo, fo;           // offsets of its rows (mtn*128) and columns (ntn*64) in the
                        // exponent and maximum arrays
  long long voff;       // element offset of its block of vectors V / W (d x m), actions
};

struct OzTiles {
  const unsigned char* px;
  const unsigned char* py;
  size_t pxs, pys;
  int mtn, ntn, kc;
  int nparts, nseg;
  int sx[2][2], sy[2][2];
  int ksplit;
  // highest digit-pair level kept, 2..8 (0 means 8): a product whose exact
  // value only matters to a coarser absolute accuracy drops levels L+1..8,
  // loads digits 1..L-1 only and issues fewer MMAs
  int lmax;
  long long* acc;  // [part][mtn*128][ntn*64][2]: hi (2^-40 units), lo (2^-64 units)
  int* err;
  // batch mode (items != nullptr): item i is tile items[i] = (b, part, mt, nt)
  // of matrix b over its whole K (ksplit 1), with the geometry and offsets of
  // mats[b]; items of matrices with mask[b] == 0 are skipped
  const int4* items;
  const BMat* mats;
  const int* mask;
  int store;       // 1: plain stores into acc (one item per tile), 0: atomic adds
  double* flops;             // batch mode: product flops (2d^3, complex 8d^3) added, nullable
  double* dflops;            // batch mode: digit-pair flops (pairs kept x product flops), nullable
  int nitems;                // work items: batch mode, the table's length; else parts x tiles x ksplit
};

// geometry of work item idx (a tile and K range) of a launch; valid = 0 for a
// masked matrix or an empty K range
struct TileGeo {
  int valid, b, part, mt, nt, kc, mtn, ntn, c0, c1, dm;
  const unsigned char* px;
  const unsigned char* py;
  size_t pxs, pys;
  long long* acc;
};

__device__ __forceinline__ TileGeo tile_geo(const OzTiles& a, int idx) {
  TileGeo G;
  G.valid = 0;
  int ks, ksplit;
  if (a.items) {
    const int4 it = a.items[idx];
    G.b = it.x;
    if (!a.mask[it.x]) return G;
    const BMat& M = a.mats[it.x];
    G.part = it.y;
    G.mt = it.z;
    G.nt = it.w;
    ks = 0;
    ksplit = 1;
    G.mtn = M.mtn;
    G.ntn = M.ntn;
    G.kc = M.kc;
    G.px = a.px + M.px;
    G.py = a.py + M.py;
    G.pxs = (size_t)G.mtn * G.kc * GXST;
    G.pys = (size_t)G.ntn * G.kc * GYST;
    G.acc = a.acc + M.acc * 2;
    G.dm = M.d;
  } else {
    int item = idx;
    G.b = 0;
    ks = item % a.ksplit;
    item /= a.ksplit;
    G.nt = item % a.ntn;
    item /= a.ntn;
    G.mt = item % a.mtn;
    G.part = item / a.mtn;
    ksplit = a.ksplit;
    G.mtn = a.mtn;
    G.ntn = a.ntn;
    G.kc = a.kc;
    G.px = a.px;
    G.py = a.py;
    G.pxs = a.pxs;
    G.pys = a.pys;
    G.acc = a.acc;
    G.dm = 1 << 30;
  }
  const int nch = a.nseg * G.kc;
  const int groups = (nch + GSTEPS - 1) / GSTEPS;
  const int gpb = (groups + ksplit - 1) / ksplit;
  const int g0 = ks * gpb, g1 = min(groups, g0 + gpb);
  if (g0 >= g1) return G;
  G.c0 = g0 * GSTEPS;
  G.c1 = min(nch, g1 * GSTEPS);
  G.valid = 1;
  return G;
}

// Persistent: CTA i takes work items i, i + gridDim.x, ... (largest first when
// the host sorts them).  Warp 16 lane 0 walks the items' K chunks with two
// cursors, one issuing bulk copies up to GNST chunks ahead (across item
// boundaries) and one issuing the MMAs; warps 0-15 read the accumulators after
// every group and write an item's sums after its last group.
static __global__ void __launch_bounds__(GTHREADS, 1) oz_tiles(OzTiles a) {
  extern __shared__ unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[GNST], empty[GNST], accf, accr;
  __shared__ uint32_t tslot;
  __shared__ int s_err;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char* smem = (unsigned char*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
  const int nitems = a.nitems;
  const int Lm = (a.lmax >= 2 && a.lmax <= 8) ? a.lmax : 8;  // levels 2..Lm
  const int nd = Lm - 1;                                    // digits used per operand

  if (tid == 0) {
    for (int i = 0; i < GNST; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(&accf, 1);
    tc::mbar_init(&accr, GRW);
    tc::mbar_fence_init();
    s_err = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tslot, oz::TMEM_COLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;

  if (warp == GRW) {
    // ---- producer and MMA issuer (one thread) ----
    if (lane == 0) {
      int err = 0;
      // load cursor (idxL, chL, GL) and MMA cursor (idxM, chM, GM)
      int idxL = blockIdx.x, idxM = blockIdx.x, chL = 0, chM = 0;
      TileGeo GL, GM;
      GL.valid = GM.valid = 0;
      while (idxL < nitems && !(GL = tile_geo(a, idxL)).valid) idxL += gridDim.x;
      if (idxL < nitems) chL = GL.c0;
      idxM = idxL;
      GM = GL;
      chM = chL;
      long long kL = 0, kM = 0;  // chunks loaded / multiplied by this CTA
      long long gcount = 0;      // groups started
      constexpr uint32_t LBO = 128, SBO = (GKC / 8) * 128;
      while (idxM < nitems && !err) {
        // keep up to GNST chunks in flight: a stage is refilled once the MMAs
        // of the chunk that used it (GNST chunks back) have finished
        while (idxL < nitems && kL < kM + GNST) {
          if (kL >= GNST && !tc::mbar_wait(&empty[kL % GNST], ((kL / GNST) - 1) & 1, oz::WAIT)) {
            err = 1;
            break;
          }
          const int s = (int)(kL % GNST);
          const int seg = chL / GL.kc, c = chL % GL.kc;
          const unsigned char* xs =
              GL.px + (size_t)a.sx[GL.part][seg] * GL.pxs + ((size_t)GL.mt * GL.kc + c) * GXST;
          const unsigned char* ys =
              GL.py + (size_t)a.sy[GL.part][seg] * GL.pys + ((size_t)GL.nt * GL.kc + c) * GYST;
          unsigned char* dst = smem + s * GST;
          tc::mbar_arrive_expect_tx(&full[s], (uint32_t)nd * (GXB + GYB));
          tc::bulk_g2s(dst, xs, (uint32_t)nd * GXB, &full[s]);
          tc::bulk_g2s(dst + GXST, ys, (uint32_t)nd * GYB, &full[s]);
          ++kL;
          if (++chL == GL.c1) {
            idxL += gridDim.x;
            while (idxL < nitems && !(GL = tile_geo(a, idxL)).valid) idxL += gridDim.x;
            if (idxL < nitems) chL = GL.c0;
          }
        }
        if (err) break;
        const int s = (int)(kM % GNST);
        const bool first = (chM % GSTEPS) == 0 || chM == GM.c0;
        if (first) {
          if (gcount > 0 && !tc::mbar_wait(&accr, (uint32_t)((gcount - 1) & 1), oz::WAIT)) {
            err = 1;
            break;
          }
          ++gcount;
        }
        if (!tc::mbar_wait(&full[s], (uint32_t)((kM / GNST) & 1), oz::WAIT)) {
          err = 1;
          break;
        }
        tc::fence_after();
        const uint32_t sx = tc::saddr(smem + s * GST);
        const uint32_t sy = sx + GXST;
#pragma unroll
        for (int p = 1; p <= oz::S; ++p) {
          if (p > nd) break;
          const uint64_t ad = tc::sdesc(sx + (p - 1) * GXB, LBO, SBO);
#pragma unroll
          for (int q0 = 1; q0 <= 8 - p; q0 += 4) {
            if (q0 > Lm - p) break;
            const int nq = min(4, Lm - p - q0 + 1);
            const uint64_t bd = tc::sdesc(sy + (q0 - 1) * GYB, LBO, SBO);
            const uint32_t id = tc::idesc_bf16(oz::TM, oz::TN * nq);
            // the first K step of a group starts every accumulator in use
            // (p = 1 covers levels 2..Lm)
            tc::mma_bf16(tmem + (p + q0 - 2) * oz::TN, ad, bd, id, (first && p == 1) ? 0u : 1u);
          }
        }
        tc::mma_commit(&empty[s]);
        ++kM;
        const bool last = ((chM + 1) % GSTEPS) == 0 || chM + 1 == GM.c1;
        if (last) tc::mma_commit(&accf);
        if (++chM == GM.c1) {
          idxM += gridDim.x;
          while (idxM < nitems && !(GM = tile_geo(a, idxM)).valid) idxM += gridDim.x;
          if (idxM < nitems) chM = GM.c0;
        }
      }
      if (err) {
        s_err = 1;
        atomicOr(a.err, 1);
      }
      // drain before TMEM is freed: every copy issued, and the last commit
      // (it covers every MMA issued before it)
      for (long long k = kM; k < kL; ++k)
        tc::mbar_wait(&full[k % GNST], (uint32_t)((k / GNST) & 1), oz::WAIT);
      if (kM > 0) tc::mbar_wait(&empty[(kM - 1) % GNST], (uint32_t)(((kM - 1) / GNST) & 1), oz::WAIT);
    }
  } else {
    // ---- readout warps ----
    const int colh = 16 * (warp >> 2);  // 16 of the tile's 64 columns per warp
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    bool ok = true;
    long long g = 0;  // groups read
    for (int idx = blockIdx.x; idx < nitems && ok; idx += gridDim.x) {
      const TileGeo G = tile_geo(a, idx);
      if (!G.valid) continue;
      if (a.flops && tid == 0 && G.part == 0 && G.mt == 0 && G.nt == 0 && G.c0 == 0) {
        const double dd = (double)G.dm;
        const double f = (a.nparts == 2 ? 8.0 : 2.0) * dd * dd * dd;
        atomicAdd(a.flops, f);
        if (a.dflops) atomicAdd(a.dflops, f * (Lm - 1) * Lm / 2);
      }
      long long ahi[16], alo[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) ahi[j] = alo[j] = 0;
      const int ng = (G.c1 - G.c0 + GSTEPS - 1) / GSTEPS;
      for (int gg = 0; gg < ng; ++gg, ++g) {
        if (!tc::mbar_wait(&accf, (uint32_t)(g & 1), oz::WAIT)) {
          ok = false;
          break;
        }
        tc::fence_after();
#pragma unroll
        for (int q = 0; q < GNACC; ++q) {
          if (q > Lm - 2) break;  // levels above Lm are not accumulated
          // level L = q + 2: value = k 2^-8L exactly with |k| < 2^24; k by the
          // FP32 -> int32 conversion (the 64-bit one runs on the FP64 unit)
          const int L = q + 2;
          const float sc = __int_as_float((127 + 8 * L) << 23);  // 2^(8L)
          uint32_t r[16];
          tc::tmem_ld16(tmem + lane_base + q * oz::TN + colh, r);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const long long k = __float2int_rz(__uint_as_float(r[j]) * sc);
            if (q < 4) ahi[j] += k << (40 - 8 * L);   // 2^-40 units
            else alo[j] += k << (64 - 8 * L);         // 2^-64 units
          }
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&accr);
      }
      if (!ok || s_err) break;
      const int Mp = G.mtn * oz::TM, Np = G.ntn * oz::TN;
      const int row = G.mt * oz::TM + 32 * (warp & 3) + lane;
      unsigned long long* dst =
          (unsigned long long*)G.acc + (((size_t)G.part * Mp + row) * Np + G.nt * oz::TN + colh) * 2;
      if (a.store) {
        // only the matrix's own rows and columns: the epilogue reads no others
        const int col0 = G.nt * oz::TN + colh;
        if (row < G.dm) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (col0 + j < G.dm) *(ulonglong2*)(dst + 2 * j) = make_ulonglong2(ahi[j], alo[j]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (ahi[j]) atomicAdd(dst + 2 * j, (unsigned long long)ahi[j]);
          if (alo[j]) atomicAdd(dst + 2 * j + 1, (unsigned long long)alo[j]);
        }
      }
    }
    if (!ok && lane == 0) atomicOr(a.err, 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, oz::TMEM_COLS);
}

}  // namespace grid
}  // namespace fmk
