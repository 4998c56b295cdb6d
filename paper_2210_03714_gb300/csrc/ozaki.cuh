// ozaki.cuh -- double-accurate products P = X Y on the 5th-generation tensor
// cores, for the refinement residuals and the squarings of the mixed
// precision path (one CTA, called from the persistent kernel).
//
// Error-free splitting (the Ozaki scheme): every row i of X is scaled by 2^-e_i
// (|x| < 2^e_i) and every column j of Y by 2^-f_j, and the scaled values are
// cut into S = 7 signed 8-bit digits,  x~ = sum_p d_p 2^(-8p),  d_1 in
// [-256, 256], d_p in [-128, 127] (p > 1), 56 bits in all.  Each digit is a
// BF16 number exactly, and so is each product of two digits; a K-long sum of
// products of digit pairs (p, q) is an integer multiple of 2^(-8(p+q)).  Pairs
// of one level L = p + q are summed in one FP32 accumulator in tensor memory:
// with K <= 128 the sum stays within 2^24 units of its level (level 8 is
// split over two accumulators to stay within it), so every FP32 accumulation
// is exact, whatever rounding the tensor core's adder applies; levels >= 9 are
// dropped (with random digits about 2^-53 of max|x| max|y| per entry, like the
// rounding of a double GEMM of this size).  Every 128 values of K the eight
// accumulators are read out and added, exactly, into two 64-bit integers:
// levels 2-5 in units of 2^-40 and levels 6-8 in units of 2^-64.  The final
// value hi 2^24 + lo (a 128-bit integer) is rounded to double once.  28
// digit-pair products replace each double product.
//
// Accuracy is relative to max_k|x_ik| max_k|y_kj| (fixed point per row and
// column), so operands with a dominant diagonal (I + E) should be passed as E.
//
// Data flow: the digits are written once per operand to global scratch in
// the tensor-core operand layout (8-row x 16-byte core matrices, K-major),
// then streamed into shared memory by bulk copies (two stages, mbarriers)
// while one thread issues tcgen05.mma into eight 128 x 64 accumulators.
#pragma once
#include <cuda_bf16.h>
#include <string.h>

#include "cta_la.cuh"
#include "tc.cuh"

namespace fmk {
namespace oz {

constexpr int S = 7;            // digits per value
constexpr int TM = 128;         // output tile rows (MMA M)
constexpr int TN = 64;          // output tile columns (MMA N)
constexpr int KC = 32;          // K per pipeline stage (two MMA K-steps)
constexpr int FLUSH = 128 / KC; // stages per exact accumulation group (K = 128)
constexpr int NACC = 8;         // accumulators: levels 2..7, and level 8 in two parts
constexpr uint32_t XBLK = TM * KC * 2;  // bytes of one digit plane of an X tile
constexpr uint32_t YBLK = TN * KC * 2;
constexpr uint32_t XSTAGE = S * XBLK;   // 57344
constexpr uint32_t YSTAGE = S * YBLK;   // 28672
constexpr uint32_t STAGE = XSTAGE + YSTAGE;
constexpr uint32_t SMEM = 2 * STAGE;    // 172032 bytes of operand staging
constexpr uint32_t TMEM_COLS = 512;
constexpr long long WAIT = 4000000000LL;  // ~2 s of clock cycles per wait

// accumulator of digit pair (p, q), 1-based digits.  Bounds at K = 128 in
// units of the level (|d_1| <= 256, |d_p| <= 128): level 2: 2^23; 3: 2^23;
// 4: 2^23 + 2^21; 5: 1.5 2^23; 6: 1.75 2^23; 7: 2^24; level 8 as
// {(1,7),(7,1),(2,6),(6,2)}: 1.5 2^23 and {(3,5),(5,3),(4,4)}: 1.5 2^22.
__host__ __device__ constexpr int acc_of(int p, int q) {
  return (p + q) <= 7 ? (p + q - 2) : ((p <= 2 || q <= 2) ? 6 : 7);
}

// scratch bytes in global memory for operands up to n x n (X) and n x m (Y)
__host__ __device__ inline size_t xs_bytes(int n, int k) {
  return (size_t)((n + TM - 1) / TM) * ((k + KC - 1) / KC) * XSTAGE;
}
__host__ __device__ inline size_t ys_bytes(int k, int m) {
  return (size_t)((m + TN - 1) / TN) * ((k + KC - 1) / KC) * YSTAGE;
}

struct Ctx {
  uint32_t* tslot;     // shared word receiving the TMEM address of each product
  uint32_t tmem;       // TMEM base address (512 columns) while a product runs
  uint64_t* bar;       // [0,1] loads of stage 0/1, [2,3] MMAs of stage 0/1
  unsigned char* smem; // SMEM bytes, 1024-aligned
  unsigned char* gx;   // digit planes of X (global)
  unsigned char* gy;   // digit planes of Y (global)
  int* ex;             // row exponents of X (global, >= M)
  int* fy;             // column exponents of Y (global, >= N)
  uint32_t use[2];     // how many times each stage buffer has been filled
  int err;             // a wait timed out
};

// byte offset of element (r, k) inside one digit plane of a tile (r < 128 or
// 64, k < KC): core matrix (r/8, k/8), K-adjacent cores 128 B apart (LBO),
// row-adjacent cores (KC/8)*128 B apart (SBO)
__device__ __forceinline__ uint32_t plane_off(int r, int k) {
  return (uint32_t)(((r >> 3) * (KC / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// The 7 digits of x * 2^-e (|x| < 2^e), as BF16 values d_p 2^(-8p).
__device__ __forceinline__ void digits(double x, int e, __nv_bfloat16* out) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long q = 0;
  if (E != 0) {  // zero or subnormal: all digits 0
    const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
    const int sh = E - 1019 - e;  // q = round(|x| 2^(56 - e))
    if (sh >= 0) q = mant << sh;
    else if (sh > -63) q = (mant + (1LL << (-sh - 1))) >> (-sh);
  }
  const bool neg = bits < 0;
  // signed digits from the bytes of q (lowest first): a byte plus the carry
  // of 128 or more becomes byte - 256 and carries one into the next byte;
  // 32-bit operations only
  const unsigned int qlo = (unsigned int)q, qhi = (unsigned int)((unsigned long long)q >> 32);
  int d[S];
  int carry = 0;
#pragma unroll
  for (int i = 0; i < S - 1; ++i) {
    const unsigned int w = i < 4 ? qlo : qhi;
    const int t = (int)((w >> (8 * (i & 3))) & 255u) + carry;
    carry = t >= 128;
    d[S - 1 - i] = t - (carry << 8);
  }
  d[0] = (int)(qhi >> 16) + carry;  // q <= 2^56 (rounding may reach 2^56): at most 256
  // d_p 2^(-8p) without conversion instructions: 1.5 2^23 + d_p is exact in
  // FP32 (|d_p| <= 256), one FMA scales it by 2^(-8p) and removes the 1.5 2^23
  // exactly, and the value (at most 8 significant bits) is its own BF16
  // truncation: the top 16 bits of the FP32 word.
#pragma unroll
  for (int p = 0; p < S; ++p) {
    const float sc = __int_as_float((127 - 8 * (p + 1)) << 23);  // 2^(-8(p+1))
    const float m = __int_as_float(0x4B400000 + (neg ? -d[p] : d[p]));
    const float f = __fmaf_rn(m, sc, -12582912.0f * sc);
    out[p] = __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
  }
}

// count of leading zero bits and a bit pattern as a double, on both sides
__host__ __device__ __forceinline__ int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}
__host__ __device__ __forceinline__ double bits_double(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
#endif
}

// m 2^e (1 <= m <= 2^53, already rounded) as a double, sign neg, assembled
// from its bits
__host__ __device__ __forceinline__ double assemble_m(unsigned long long m, int e, bool neg) {
  const int nbm = 64 - clz64(m);
  const int ef = e + nbm - 1 + 1023;  // biased exponent of the result
  const unsigned long long sgn = neg ? 0x8000000000000000ULL : 0ULL;
  const unsigned long long mant = nbm <= 53 ? (m << (53 - nbm)) : (m >> (nbm - 53));
  if (ef >= 1 && ef <= 2046)
    return bits_double(((unsigned long long)ef << 52) | (mant & 0xFFFFFFFFFFFFFULL) | sgn);
  // outside the normal range, with integer operations only (no FP64 unit):
  // overflow to infinity; below 2^-1022 the 53-bit mantissa is shifted into
  // the subnormal field (truncated: such values are far below any result here)
  if (ef > 2046) return bits_double(sgn | 0x7FF0000000000000ULL);
  const int sh = 1 - ef;
  return bits_double(sgn | (sh < 64 ? (mant >> sh) : 0ULL));
}

// round-to-nearest double of v 2^e2, v an exact 128-bit integer
__host__ __device__ __forceinline__ double round_i128(__int128 v, int e2) {
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long ah = (unsigned long long)(a >> 64), al = (unsigned long long)a;
  const int nb = ah ? 128 - clz64(ah) : 64 - clz64(al);  // bit length
  unsigned long long m;
  int e = e2;
  if (nb <= 53) {
    m = al;
  } else {
    const int sh = nb - 53;
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    const unsigned __int128 rem = a & (((unsigned __int128)1 << sh) - 1);
    m = (unsigned long long)(a >> sh);
    if (rem > half || (rem == half && (m & 1))) m += 1;
    e += sh;
  }
  return assemble_m(m, e, neg);
}

// t 2^e rounded to nearest (ties to even), t nonzero and below 2^63, sticky:
// nonzero bits below t's lowest bit were dropped (never on a tie then)
__host__ __device__ __forceinline__ double round_u64(unsigned long long t, bool sticky, int e,
                                                     bool neg) {
  const int nb = 64 - clz64(t);
  unsigned long long m = t;
  if (nb > 53) {
    const int sh = nb - 53;
    const unsigned long long half = 1ULL << (sh - 1);
    const unsigned long long rem = t & ((1ULL << sh) - 1);
    m = t >> sh;
    if (rem > half || (rem == half && (sticky || (m & 1)))) m += 1;
    e += sh;
  }
  return assemble_m(m, e, neg);
}

// The same rounding of (hi 2^24 + lo) 2^e2 as round_i128, for the two exact
// sums of the tile products (|hi|, |lo| < 2^62), with 64-bit operations only:
// hi 2^24 + lo = s 2^24 + l, s = hi + floor(lo / 2^24), 0 <= l < 2^24; when
// |s| < 2^39 the value is a 63-bit integer, else its top 63 bits are kept and
// the rest of l folded into a sticky bit (the rounding position is then at
// bit 10 or above, so no tie is lost).
__host__ __device__ __forceinline__ double round_hl(long long hi, long long lo, int e2) {
  const long long s1 = hi + (lo >> 24);  // arithmetic shift: floor
  unsigned long long l0 = (unsigned long long)lo & 0xFFFFFFULL;
  const bool neg = s1 < 0;
  unsigned long long m1 = (unsigned long long)s1;
  if (neg) {  // |value| = (-s1) 2^24 - l0
    m1 = 0ULL - m1;
    if (l0) {
      m1 -= 1;
      l0 = (1ULL << 24) - l0;
    }
  }
  if (m1 < (1ULL << 39)) {  // |value| = m1 2^24 + l0 < 2^63
    const unsigned long long t = (m1 << 24) | l0;
    return t ? round_u64(t, false, e2, neg) : 0.0;
  }
  const int k = (64 - clz64(m1)) - 39;  // 1 .. 23: keep the top 63 bits
  const unsigned long long t = (m1 << (24 - k)) | (l0 >> k);
  return round_u64(t, (l0 & ((1ULL << k) - 1)) != 0, e2 + k, neg);
}

// s 2^k z as an exact multiple of 2^e (z double, s = +-1): false when z is not
// finite or the value would need more than 126 bits; bits of z below 2^e are
// rounded to nearest (at most half a unit 2^e)
__device__ __forceinline__ bool to_fixed(double z, int k, bool neg, int e, __int128& out) {
  const long long bits = __double_as_longlong(z);
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0x7FF) return false;
  if (E == 0) {  // zero or subnormal: below every unit these sums use
    out = 0;
    return true;
  }
  const long long m = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const int sh = E - 1075 + k - e;  // s 2^k z = +-m 2^(sh + e)
  __int128 v;
  if (sh >= 0) {
    if (sh > 72) return false;
    v = (__int128)m << sh;
  } else if (sh > -60) {
    v = (m + (1LL << (-sh - 1))) >> (-sh);
  } else {
    v = 0;
  }
  out = ((bits < 0) != neg) ? -v : v;
  return true;
}

// round-to-nearest double of (hi 2^24 + lo) 2^e2, hi and lo exact integers
// (|hi|, |lo| < 2^62)
__host__ __device__ __forceinline__ double combine_scaled(long long hi, long long lo, int e2) {
  return round_hl(hi, lo, e2);
}


// exponent e with |x| < 2^e from the bit pattern of the largest |x| (0 for an
// all-zero set; integer operations only):
// 1.f 2^(E - 1023) < 2^(E - 1022); subnormals < 2^-1022
__device__ __forceinline__ int exp_above_bits(unsigned long long b) {
  if (b == 0) return 0;
  const int E = (int)(b >> 52);
  return E == 0 ? -1022 : E - 1022;
}

// Split X (M x K, row-major, ld) row-wise into digit planes in ctx.gx.
static __device__ void split_rows(Ctx& c, int M, int K, const double* X, int ldx, double* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int mt = (M + TM - 1) / TM, kc = (K + KC - 1) / KC;
  for (int r = warp; r < mt * TM; r += NT / 32) {
    unsigned long long mx = 0;  // largest |x| as bits: integer operations only
    if (r < M)
      for (int k = lane; k < K; k += 32) {
        const unsigned long long b =
            (unsigned long long)__double_as_longlong(X[(size_t)r * ldx + k]) & 0x7FFFFFFFFFFFFFFFULL;
        mx = b > mx ? b : mx;
      }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = b > mx ? b : mx;
    }
    if (lane == 0) c.ex[r] = exp_above_bits(mx);
  }
  __syncthreads();
  // work item: one row, 8 consecutive k -> 7 x 16-byte stores
  const int items = mt * TM * kc * (KC / 8);
  for (int it = tid; it < items; it += NT) {
    const int k8 = it % (kc * (KC / 8));
    const int r = it / (kc * (KC / 8));
    const int e = c.ex[r];
    __align__(16) __nv_bfloat16 dig[S][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k8 * 8 + j;
      const double x = (r < M && k < K) ? X[(size_t)r * ldx + k] : 0.0;
      __nv_bfloat16 t[S];
      digits(x, e, t);
#pragma unroll
      for (int p = 0; p < S; ++p) dig[p][j] = t[p];
    }
    const int tile = r / TM, chunk = (k8 * 8) / KC;
    unsigned char* base = c.gx + ((size_t)tile * kc + chunk) * XSTAGE;
    const uint32_t off = plane_off(r % TM, (k8 * 8) % KC);
#pragma unroll
    for (int p = 0; p < S; ++p) *(uint4*)(base + p * XBLK + off) = *(const uint4*)dig[p];
  }
  (void)red;
}

// Split Y (K x N, row-major, ld) column-wise into digit planes in ctx.gy
// (stored N-major: the B operand of the MMA is K-major).
static __device__ void split_cols(Ctx& c, int K, int N, const double* Y, int ldy) {
  const int tid = threadIdx.x;
  const int nt = (N + TN - 1) / TN, kc = (K + KC - 1) / KC;
  for (int j = tid; j < nt * TN; j += NT) {
    unsigned long long mx = 0;
    if (j < N) {
#pragma unroll 8
      for (int k = 0; k < K; ++k) {
        const unsigned long long b =
            (unsigned long long)__double_as_longlong(Y[(size_t)k * ldy + j]) & 0x7FFFFFFFFFFFFFFFULL;
        mx = b > mx ? b : mx;
      }
    }
    c.fy[j] = exp_above_bits(mx);
  }
  __syncthreads();
  const int items = nt * TN * kc * (KC / 8);
  for (int it = tid; it < items; it += NT) {
    const int j = it % (nt * TN);
    const int k8 = it / (nt * TN);
    const int e = c.fy[j];
    __align__(16) __nv_bfloat16 dig[S][8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int k = k8 * 8 + jj;
      const double y = (j < N && k < K) ? Y[(size_t)k * ldy + j] : 0.0;
      __nv_bfloat16 t[S];
      digits(y, e, t);
#pragma unroll
      for (int p = 0; p < S; ++p) dig[p][jj] = t[p];
    }
    const int tile = j / TN, chunk = (k8 * 8) / KC;
    unsigned char* base = c.gy + ((size_t)tile * kc + chunk) * YSTAGE;
    const uint32_t off = plane_off(j % TN, (k8 * 8) % KC);
#pragma unroll
    for (int p = 0; p < S; ++p) *(uint4*)(base + p * YBLK + off) = *(const uint4*)dig[p];
  }
}

// issue the bulk copies of chunk `chunk` of tile (mt, nt) into stage s
__device__ __forceinline__ void load_stage(Ctx& c, int s, int mt, int nt, int chunk, int kc) {
  uint64_t* lb = c.bar + s;
  unsigned char* dst = c.smem + s * STAGE;
  tc::mbar_arrive_expect_tx(lb, STAGE);
  tc::bulk_g2s(dst, c.gx + ((size_t)mt * kc + chunk) * XSTAGE, XSTAGE, lb);
  tc::bulk_g2s(dst + XSTAGE, c.gy + ((size_t)nt * kc + chunk) * YSTAGE, YSTAGE, lb);
}

// the 28 digit-pair MMAs of one stage (two K=16 steps each)
__device__ __forceinline__ void mma_stage(Ctx& c, int s, bool first_in_group) {
  const uint32_t sx = tc::saddr(c.smem + s * STAGE);
  const uint32_t sy = sx + XSTAGE;
  constexpr uint32_t idesc = tc::idesc_bf16(TM, TN);
  bool fresh[NACC];
#pragma unroll
  for (int a = 0; a < NACC; ++a) fresh[a] = first_in_group;
#pragma unroll
  for (int p = 1; p <= S; ++p)
#pragma unroll
    for (int q = 1; q <= S; ++q) {
      if (p + q > 8) continue;
      const int a = acc_of(p, q);
#pragma unroll
      for (int ks = 0; ks < KC / 16; ++ks) {
        const uint64_t ad = tc::sdesc(sx + (p - 1) * XBLK + ks * 256, 128, (KC / 8) * 128);
        const uint64_t bd = tc::sdesc(sy + (q - 1) * YBLK + ks * 256, 128, (KC / 8) * 128);
        tc::mma_bf16(c.tmem + a * TN, ad, bd, idesc, fresh[a] ? 0u : 1u);
        fresh[a] = false;
      }
    }
}

// P (M x N) = X (M x K) Y (K x N), all double, row-major.  All NT threads.
// Returns 0, or 1 when a wait timed out (P is then not valid).
// reuse_x: X is the operand of the previous call (its digit planes are kept)
static __device__ __noinline__ int gemm(Ctx& c, int M, int N, int K, const double* X, int ldx,
                                 const double* Y, int ldy, double* P, int ldp,
                                 bool reuse_x = false) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (!reuse_x) split_rows(c, M, K, X, ldx, nullptr);
  split_cols(c, K, N, Y, ldy);
  tc::fence_proxy_async();
  __syncthreads();
  const int mtn = (M + TM - 1) / TM, ntn = (N + TN - 1) / TN, kc = (K + KC - 1) / KC;
  const int row = 32 * (warp & 3) + lane;  // TMEM lane this thread reads
  const int colh = 32 * (warp >> 2);       // first of its 32 tile columns
  __shared__ int s_err;
  if (tid == 0) s_err = c.err;
  // tensor memory for this product only: all 512 columns in one request, so
  // a CTA waiting for it never holds part of it (two CTAs share an SM)
  if (warp == 0) tc::tmem_alloc(c.tslot, TMEM_COLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (tid == 0) c.tmem = *c.tslot;
  __syncthreads();
  for (int mt = 0; mt < mtn; ++mt)
    for (int nt = 0; nt < ntn; ++nt) {
      long long ahi[32], alo[32];  // levels 2-5 (units 2^-40), 6-8 (units 2^-64)
#pragma unroll
      for (int j = 0; j < 32; ++j) ahi[j] = alo[j] = 0;
      for (int g0 = 0; g0 < kc; g0 += FLUSH) {
        const int g1 = min(kc, g0 + FLUSH);
        if (tid == 0 && !s_err) {
          // stage s holds chunk (ch % 2); before refilling it, the MMAs of the
          // chunk that used it last must be done (their commit on bar[2 + s])
          for (int ch = g0; ch < g1; ++ch) {
            const int s = ch & 1;
            if (ch == g0) {
              load_stage(c, s, mt, nt, ch, kc);
              c.use[s] += 1;
            }
            if (!tc::mbar_wait(c.bar + s, (c.use[s] - 1) & 1, WAIT)) { s_err = 1; break; }
            tc::fence_after();
            mma_stage(c, s, ch == g0);
            tc::mma_commit(c.bar + 2 + s);
            if (ch + 1 < g1) {
              const int s2 = (ch + 1) & 1;
              // the other stage: wait for the MMAs that read it (chunk ch - 1)
              if (ch > g0 && !tc::mbar_wait(c.bar + 2 + s2, (c.use[s2] - 1) & 1, WAIT)) {
                s_err = 1;
                break;
              }
              load_stage(c, s2, mt, nt, ch + 1, kc);
              c.use[s2] += 1;
            }
          }
          // every MMA of the group is covered by the last commit
          const int sl = (g1 - 1) & 1;
          if (!s_err && !tc::mbar_wait(c.bar + 2 + sl, (c.use[sl] - 1) & 1, WAIT)) s_err = 1;
          // the other stage's last commit (if used in this group) completed earlier
          if (!s_err && g1 - g0 > 1) {
            const int so = sl ^ 1;
            if (!tc::mbar_wait(c.bar + 2 + so, (c.use[so] - 1) & 1, WAIT)) s_err = 1;
          }
        }
        __syncthreads();
        tc::fence_after();
        if (!s_err) {
          // read the eight accumulators of this group into the two exact sums
#pragma unroll 1
          for (int a = 0; a < NACC; ++a) {
            uint32_t r[32];
            tc::tmem_ld32(c.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + a * TN + colh, r);
            tc::tmem_ld_wait();
            // accumulator a holds an exact multiple of 2^-8L (L = a + 2, level 8
            // for a = 6, 7): its integer, shifted to the unit of its sum
            const int L = a < 6 ? a + 2 : 8;
            // k = value 2^(8L), |k| < 2^24, by the FP32 -> int32 conversion
            const float sc = __int_as_float((127 + 8 * L) << 23);
            if (a < 4) {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                ahi[j] += (long long)__float2int_rz(__uint_as_float(r[j]) * sc) << (40 - 8 * L);
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                alo[j] += (long long)__float2int_rz(__uint_as_float(r[j]) * sc) << (64 - 8 * L);
            }
          }
        }
        tc::fence_before();
        __syncthreads();
      }
      // P = (hi 2^24 + lo) 2^(e_i + f_j - 64), rounded once
      const int i = mt * TM + row;
      if (!s_err && i < M) {
        const int ei = c.ex[i];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int jj = nt * TN + colh + j;
          if (jj < N) P[(size_t)i * ldp + jj] = combine_scaled(ahi[j], alo[j], ei + c.fy[jj] - 64);
        }
      }
      __syncthreads();
    }
  const int err = s_err;
  if (tid == 0) {
    c.err = err;
    if (err) {  // let copies and MMAs still in flight finish before freeing
      for (int st = 0; st < 2; ++st)
        if (c.use[st]) {
          tc::mbar_wait(c.bar + st, (c.use[st] - 1) & 1, WAIT);
          tc::mbar_wait(c.bar + 2 + st, (c.use[st] - 1) & 1, WAIT);
        }
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(c.tmem, TMEM_COLS);
  __syncthreads();
  return err;
}

}  // namespace oz
}  // namespace fmk
