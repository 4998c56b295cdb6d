// fm_launch.cu -- dispatch to the per-type kernels, and the batch-ordering kernel.
#include "fm_kernels.cuh"
#include "fm_launch.h"

namespace fmk {

size_t launch_smem(bool cplx, int nb, int dmax, bool tck) {
  if (cplx) return nb == 16 ? fm_smem_bytes<zd, 16>(dmax) : fm_smem_bytes<zd, 8>(dmax);
  return nb == 16 ? fm_smem_bytes<double, 16>(dmax, tck) : fm_smem_bytes<double, 8>(dmax, tck);
}

int launch_occupancy(bool cplx, int precision, int nb, size_t smem) {
  return cplx ? occ_cplx(precision, nb, smem) : occ_real(precision, nb, smem);
}

cudaError_t launch_persistent(bool cplx, int precision, int nb, const FmJob& J, const FmCoef& cf,
                              int grid, size_t smem, cudaStream_t st) {
  return cplx ? launch_cplx(precision, nb, J, cf, grid, smem, st)
              : launch_real(precision, nb, J, cf, grid, smem, st);
}

// Counting sort of the batch by d, largest first (longest jobs start first so
// the persistent CTAs finish together).  Matrices with d outside [1, dmax] get
// info = -4 and are left out of the queue; matrices with d in [1, dmax] but
// outside [lo, hi] belong to another part of a split batch and are left out
// without a status.
__global__ void fm_order_kernel(const int* __restrict__ d, int batch, int dmax, int lo, int hi,
                                int* order, int* counter, int* info) {
  extern __shared__ int hist[];
  for (int i = threadIdx.x; i <= dmax; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    const int dd = d[b];
    if (dd >= 1 && dd <= dmax) {
      if (dd >= lo && dd <= hi) atomicAdd(&hist[dmax - dd], 1);
    } else if (info) {
      info[b] = -4;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int i = 0; i <= dmax; ++i) {
      const int c = hist[i];
      hist[i] = run;
      run += c;
    }
    counter[0] = 0;
    counter[1] = run;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    const int dd = d[b];
    if (dd >= 1 && dd <= dmax && dd >= lo && dd <= hi) order[atomicAdd(&hist[dmax - dd], 1)] = b;
  }
}

// Step a1 alone: eta = ||t_b A_b||_1 (column sums of |t a| with the rows in
// ascending order, as every path forms them) or anorm |t_b|; then s (smallest
// s >= 0 with eta / 2^s <= theta) or N = max(1, ceil(eta / theta)).  One block
// per matrix.
template <class T>
__global__ void fm_select_kernel(const int* __restrict__ d, const int64_t* __restrict__ off,
                                 const T* __restrict__ A, const double* __restrict__ t, int dmax,
                                 double anorm, double theta, int steps, long long fixed,
                                 long long* out, int* info) {
  __shared__ double red[32];
  using TT = Tr<T>;
  const int b = blockIdx.x, tid = threadIdx.x;
  const int n = d[b];
  if (n < 1 || n > dmax) {
    if (tid == 0) {
      info[b] = -4;
      out[b] = 0;
    }
    return;
  }
  const T* Ab = A + off[b];
  const double tb = t[b];
  int bad = !isfinite(tb);
  double cmax = 0;
  for (int c = tid; c < n; c += blockDim.x) {
    double sc = 0;
    for (int r = 0; r < n; ++r) {
      const T a = Ab[(size_t)r * n + c];
      bad |= !TT::finite(a);
      sc += (double)TT::mag(TT::rscale(a, tb));
    }
    cmax = (sc > cmax || isnan(sc)) ? sc : cmax;
  }
  bad = __syncthreads_or(bad);
  for (int o = 16; o; o >>= 1) {
    const double v = __shfl_xor_sync(0xffffffffu, cmax, o);
    cmax = (v > cmax || isnan(v)) ? v : cmax;
  }
  if ((tid & 31) == 0) red[tid >> 5] = cmax;
  __syncthreads();
  if (tid == 0) {
    double m = 0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) m = (red[w] > m || isnan(red[w])) ? red[w] : m;
    const double eta = anorm > 0 ? anorm * fabs(tb) : m;
    long long v;
    if (fixed > 0 || (!steps && fixed == 0)) {
      v = fixed;
    } else if (steps) {
      const double qn = ceil(eta / theta);
      v = qn < 1.0 ? 1 : (long long)qn;
    } else {
      int s = 0;
      while (eta > ldexp(theta, s) && s < 1023) ++s;
      v = s;
    }
    out[b] = v;
    info[b] = bad ? -2 : 0;
  }
}

cudaError_t launch_select(bool cplx, const int* d, const int64_t* off, const void* A,
                          const double* t, int batch, int dmax, double anorm, double theta,
                          int steps, long long fixed, long long* out, int* info, cudaStream_t st) {
  if (cplx)
    fm_select_kernel<zd><<<batch, 256, 0, st>>>(d, off, (const zd*)A, t, dmax, anorm, theta, steps,
                                                fixed, out, info);
  else
    fm_select_kernel<double><<<batch, 256, 0, st>>>(d, off, (const double*)A, t, dmax, anorm, theta,
                                                    steps, fixed, out, info);
  return cudaGetLastError();
}

// probe matrices for the autotuner: entries from a counter hash (SplitMix64),
// uniform in [-1, 1), times scale
__global__ void fm_probe_fill(double* A, long long count, unsigned long long seed, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    A[i] = scale * ((double)(z >> 11) * 0x1.0p-52 - 1.0);
  }
}

cudaError_t launch_probe_fill(double* A, long long count, unsigned long long seed, double scale,
                              cudaStream_t st) {
  fm_probe_fill<<<1024, 256, 0, st>>>(A, count, seed, scale);
  return cudaGetLastError();
}

cudaError_t launch_order(const int* d, int batch, int dmax, int lo, int hi, int* order,
                         int* counter, int* info, cudaStream_t st) {
  fm_order_kernel<<<1, 1024, (size_t)(dmax + 1) * sizeof(int), st>>>(d, batch, dmax, lo, hi,
                                                                       order, counter, info);
  return cudaGetLastError();
}

}  // namespace fmk
