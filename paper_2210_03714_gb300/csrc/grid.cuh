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

// (cr + i ci) * a with one rounding per real operation (real: cr * a)
template <class T> __device__ __forceinline__ T cmul(double cr, double ci, T a);
template <> __device__ __forceinline__ double cmul<double>(double cr, double, double a) {
  return __dmul_rn(cr, a);
}
template <> __device__ __forceinline__ zd cmul<zd>(double cr, double ci, zd a) {
  return Tr<zd>::mul(zd{cr, ci}, a);
}

__device__ __forceinline__ void max_bits(unsigned long long* dst, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(dst, (unsigned long long)__double_as_longlong(v));
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
__global__ void colsum_max(int n, const double* colsum, double* eta) {
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
};

template <class T>
__global__ void epilogue(int M, int N, const long long* acc, int parts, int Mp, int Np,
                         const int* ex, const int* fy, const T* Pd, int ldp, Epi e, T* out,
                         int ldo) {
  const size_t count = (size_t)M * N;
  double mx = 0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count;
       k += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(k / N), j = (int)(k % N);
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
    T v = cmul<T>(e.ar, e.ai, El<T>::make(pr, pi));
    if (e.Z1) v = Tr<T>::add(v, cmul<T>(e.b1r, e.b1i, ((const T*)e.Z1)[(size_t)i * e.ld1 + j]));
    if (e.Z2) v = Tr<T>::add(v, cmul<T>(e.b2r, e.b2i, ((const T*)e.Z2)[(size_t)i * e.ld2 + j]));
    if (i == j && (e.gr != 0 || e.gi != 0)) v = Tr<T>::add(v, El<T>::make(e.gr, e.gi));
    out[(size_t)i * ldo + j] = v;
    mx = fmax(mx, fmax(fabs(El<T>::re(v)), fabs(El<T>::im(v))));
  }
  if (e.maxabs) {
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) max_bits(e.maxabs, mx);
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
// Digit planes in global memory, in the layout of ozaki.cuh: for plane set s,
// row tile mt (128 rows) and K chunk c (32 values), XSTAGE bytes at
//   px + s * pxs + (mt * kc + c) * XSTAGE
// (7 planes of 128 x 32 BF16 in 8 x 16-byte core matrices), likewise Y with
// column tiles of 64.  A complex operand has sets (re, im) for X and
// (re, im, -im) for Y, all sharing one exponent per row (column).

// largest |re|, |im| of every row of X (bits, dst zeroed by the caller)
template <class T>
__global__ void row_max(int M, int K, const T* X, int ldx, unsigned long long* rmax) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = w; r < M; r += nw) {
    double mx = 0;
    for (int k = lane; k < K; k += 32) {
      const T v = X[(size_t)r * ldx + k];
      mx = fmax(mx, fmax(fabs(El<T>::re(v)), fabs(El<T>::im(v))));
    }
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) rmax[r] = (unsigned long long)__double_as_longlong(mx);
  }
}

// largest |re|, |im| of every column of Y: blocks of 32 columns x 8 row lanes
template <class T>
__global__ void col_max(int K, int N, const T* Y, int ldy, unsigned long long* cmax) {
  __shared__ double red[8][33];
  const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + cx;
  double mx = 0;
  if (j < N)
    for (int k = blockIdx.y * 8 + ry; k < K; k += 8 * gridDim.y) {
      const T v = Y[(size_t)k * ldy + j];
      mx = fmax(mx, fmax(fabs(El<T>::re(v)), fabs(El<T>::im(v))));
    }
  red[ry][cx] = mx;
  __syncthreads();
  if (ry == 0 && j < N) {
    for (int q = 1; q < 8; ++q) mx = fmax(mx, red[q][cx]);
    max_bits(cmax + j, mx);
  }
}

__device__ __forceinline__ int exp_of_bits(unsigned long long b) {
  return oz::exp_above(__longlong_as_double((long long)b));
}

// X (M x K) -> row digit planes; item = (row, 8 consecutive k)
template <class T>
__global__ void split_rows(int M, int K, const T* X, int ldx, const unsigned long long* rmax,
                           unsigned char* px, size_t pxs, int kc, int* ex) {
  const int mtn = (M + oz::TM - 1) / oz::TM;
  const long long items = (long long)mtn * oz::TM * kc * (oz::KC / 8);
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int k8 = (int)(it % (kc * (oz::KC / 8)));
    const int r = (int)(it / (kc * (oz::KC / 8)));
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
    const int tile = r / oz::TM, chunk = (k8 * 8) / oz::KC;
    const size_t blk = ((size_t)tile * kc + chunk) * oz::XSTAGE;
    const uint32_t off = oz::plane_off(r % oz::TM, (k8 * 8) % oz::KC);
#pragma unroll
    for (int p = 0; p < oz::S; ++p) *(uint4*)(px + blk + p * oz::XBLK + off) = *(const uint4*)dr[p];
    if (El<T>::parts == 2) {
#pragma unroll
      for (int p = 0; p < oz::S; ++p)
        *(uint4*)(px + pxs + blk + p * oz::XBLK + off) = *(const uint4*)di[p];
    }
  }
}

// Y (K x N) -> column digit planes (N-major); item = (column, 8 consecutive k)
template <class T>
__global__ void split_cols(int K, int N, const T* Y, int ldy, const unsigned long long* cmax,
                           unsigned char* py, size_t pys, int kc, int* fy) {
  const int ntn = (N + oz::TN - 1) / oz::TN;
  const long long items = (long long)ntn * oz::TN * kc * (oz::KC / 8);
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
    const int tile = j / oz::TN, chunk = (k8 * 8) / oz::KC;
    const size_t blk = ((size_t)tile * kc + chunk) * oz::YSTAGE;
    const uint32_t off = oz::plane_off(j % oz::TN, (k8 * 8) % oz::KC);
#pragma unroll
    for (int p = 0; p < oz::S; ++p) *(uint4*)(py + blk + p * oz::YBLK + off) = *(const uint4*)dr[p];
    if (El<T>::parts == 2) {
#pragma unroll
      for (int p = 0; p < oz::S; ++p) {
        *(uint4*)(py + pys + blk + p * oz::YBLK + off) = *(const uint4*)di[p];
        *(uint4*)(py + 2 * pys + blk + p * oz::YBLK + off) = *(const uint4*)dn[p];
      }
    }
  }
}

// One work item per CTA: output tile (mt, nt) of part `part` over a range of
// exact accumulation groups (128 values of the concatenated K).  The part's
// K runs over nseg segments, segment g pairing X plane set sx[part][g] with Y
// plane set sy[part][g] (complex: re = Xr Yr + Xi (-Yi), im = Xr Yi + Xi Yr).
struct OzTiles {
  const unsigned char* px;
  const unsigned char* py;
  size_t pxs, pys;
  int mtn, ntn, kc;
  int nparts, nseg;
  int sx[2][2], sy[2][2];
  int ksplit;
  long long* acc;  // [part][mtn*128][ntn*64][2]: hi (2^-40 units), lo (2^-64 units)
  int* err;
};

__global__ void __launch_bounds__(NT, 1) oz_tiles(OzTiles a) {
  extern __shared__ unsigned char dsm[];
  __shared__ __align__(8) uint64_t bar[4];
  __shared__ uint32_t tslot;
  __shared__ int s_err;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char* smem = (unsigned char*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
  int item = blockIdx.x;
  const int ks = item % a.ksplit;
  item /= a.ksplit;
  const int nt = item % a.ntn;
  item /= a.ntn;
  const int mt = item % a.mtn;
  const int part = item / a.mtn;
  const int nch = a.nseg * a.kc;
  const int groups = (nch + oz::FLUSH - 1) / oz::FLUSH;
  const int gpb = (groups + a.ksplit - 1) / a.ksplit;
  const int g0 = ks * gpb, g1 = min(groups, g0 + gpb);
  if (g0 >= g1) return;  // the whole CTA leaves before any barrier or allocation

  if (tid == 0) {
    for (int i = 0; i < 4; ++i) tc::mbar_init(&bar[i], 1);
    tc::mbar_fence_init();
    s_err = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tslot, oz::TMEM_COLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  uint32_t use0 = 0, use1 = 0;  // fills of each stage (thread 0)
  auto use = [&](int s) -> uint32_t { return s ? use1 : use0; };
  auto load = [&](int s, int ch) {
    const int seg = ch / a.kc, c = ch % a.kc;
    const unsigned char* xs =
        a.px + (size_t)a.sx[part][seg] * a.pxs + ((size_t)mt * a.kc + c) * oz::XSTAGE;
    const unsigned char* ys =
        a.py + (size_t)a.sy[part][seg] * a.pys + ((size_t)nt * a.kc + c) * oz::YSTAGE;
    unsigned char* dst = smem + s * oz::STAGE;
    tc::mbar_arrive_expect_tx(&bar[s], oz::STAGE);
    tc::bulk_g2s(dst, xs, oz::XSTAGE, &bar[s]);
    tc::bulk_g2s(dst + oz::XSTAGE, ys, oz::YSTAGE, &bar[s]);
    if (s) ++use1; else ++use0;
  };
  auto mma = [&](int s, bool first) {
    const uint32_t sx = tc::saddr(smem + s * oz::STAGE);
    const uint32_t sy = sx + oz::XSTAGE;
    constexpr uint32_t idesc = tc::idesc_bf16(oz::TM, oz::TN);
    bool fresh[oz::NACC];
#pragma unroll
    for (int q = 0; q < oz::NACC; ++q) fresh[q] = first;
#pragma unroll
    for (int p = 1; p <= oz::S; ++p)
#pragma unroll
      for (int q = 1; q <= oz::S; ++q) {
        if (p + q > 8) continue;
        const int ac = oz::acc_of(p, q);
#pragma unroll
        for (int k16 = 0; k16 < oz::KC / 16; ++k16) {
          const uint64_t ad = tc::sdesc(sx + (p - 1) * oz::XBLK + k16 * 256, 128, (oz::KC / 8) * 128);
          const uint64_t bd = tc::sdesc(sy + (q - 1) * oz::YBLK + k16 * 256, 128, (oz::KC / 8) * 128);
          tc::mma_bf16(tmem + ac * oz::TN, ad, bd, idesc, fresh[ac] ? 0u : 1u);
          fresh[ac] = false;
        }
      }
  };

  long long ahi[32], alo[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) ahi[j] = alo[j] = 0;
  const int colh = 32 * (warp >> 2);
  for (int g = g0; g < g1; ++g) {
    const int c0 = g * oz::FLUSH, c1 = min(nch, c0 + oz::FLUSH);
    if (tid == 0 && !s_err) {
      // chunk ch uses stage ch & 1; the first chunk of a group is loaded here,
      // the next one while the MMAs of the current chunk run
      for (int ch = c0; ch < c1; ++ch) {
        const int s = ch & 1;
        if (ch == c0) load(s, ch);
        if (!tc::mbar_wait(&bar[s], (use(s) - 1) & 1, oz::WAIT)) { s_err = 1; break; }
        tc::fence_after();
        mma(s, ch == c0);
        tc::mma_commit(&bar[2 + s]);
        if (ch + 1 < c1) {
          const int s2 = (ch + 1) & 1;
          if (ch > c0 && !tc::mbar_wait(&bar[2 + s2], (use(s2) - 1) & 1, oz::WAIT)) { s_err = 1; break; }
          load(s2, ch + 1);
        }
      }
      const int sl = (c1 - 1) & 1;
      if (!s_err && !tc::mbar_wait(&bar[2 + sl], (use(sl) - 1) & 1, oz::WAIT)) s_err = 1;
      if (!s_err && c1 - c0 > 1 && !tc::mbar_wait(&bar[2 + (sl ^ 1)], (use(sl ^ 1) - 1) & 1, oz::WAIT))
        s_err = 1;
    }
    __syncthreads();
    tc::fence_after();
    if (!s_err) {
#pragma unroll 1
      for (int q = 0; q < oz::NACC; ++q) {
        uint32_t r[32];
        tc::tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + q * oz::TN + colh, r);
        tc::tmem_ld_wait();
        const int L = q < 6 ? q + 2 : 8;
        if (q < 4) {
#pragma unroll
          for (int j = 0; j < 32; ++j) ahi[j] += (long long)oz::exact_int(r[j], 8 * L) << (40 - 8 * L);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) alo[j] += (long long)oz::exact_int(r[j], 8 * L) << (64 - 8 * L);
        }
      }
    }
    tc::fence_before();
    __syncthreads();
  }
  if (!s_err) {
    const int Mp = a.mtn * oz::TM, Np = a.ntn * oz::TN;
    const int row = mt * oz::TM + 32 * (warp & 3) + lane;
    unsigned long long* dst =
        (unsigned long long*)a.acc + (((size_t)part * Mp + row) * Np + nt * oz::TN + colh) * 2;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (ahi[j]) atomicAdd(dst + 2 * j, (unsigned long long)ahi[j]);
      if (alo[j]) atomicAdd(dst + 2 * j + 1, (unsigned long long)alo[j]);
    }
  }
  if (tid == 0 && s_err) {
    atomicOr(a.err, 1);
    // let copies and MMAs still in flight finish before the memory is freed
    for (int s = 0; s < 2; ++s)
      if (use(s)) {
        tc::mbar_wait(&bar[s], (use(s) - 1) & 1, oz::WAIT);
        tc::mbar_wait(&bar[2 + s], (use(s) - 1) & 1, oz::WAIT);
      }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, oz::TMEM_COLS);
}

}  // namespace grid
}  // namespace fmk
