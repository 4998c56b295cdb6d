/*
 * fm.h -- C ABI of libfm: functions of matrices, and their action on blocks of
 * vectors, as a fixed linear combination of k independent shifted solves.
 *
 * Method: S. Blanes, "Parallel computation of functions of matrices and their
 * action on vectors", arXiv:2210.03714.
 *   r(x) = a0 + d1 x + d2 x^2 + sum_i b_i c_i x / (1 - c_i x)      (Eq. ParallRoundOff,
 *                                                                 Eq. Frac10R)
 *   r(x) = d0 + d1 x + d2 x^2 + sum_i b_i / (1 - c_i x)           (Eq. rat1, ParallHybrid)
 * with d0 = a0 - sum_i b_i; each term needs one solve with M_i = I - c_i B
 * (Sec. 2: the "processors" F_i = (I - c_i B)^{-1}).  f(tA) is r(B)^(2^s) with
 * B = tA/2^s (Sec. 1, scaling and squaring); f(tA)V is N steps V <- r(B)V with
 * B = tA/N and each factorization done once (Sec. 1; Sec. 5.1 remarks);
 * phi_1 uses the doubling phi1(2X) = (e^X + I) phi1(X) / 2 (Sec. 1).
 * s (or N) is the smallest value with ||B||_1 <= theta, theta from the forward
 * error bound of Sec. 3.
 *
 * Conventions for every entry point below:
 *  - Matrices are dense, row-major, with a leading dimension (elements between
 *    consecutive rows, >= number of columns).  Real data is double; complex data
 *    ("z" functions) is interleaved (re, im) double pairs.
 *  - A, V, F, W, Phi, E, t_dev, d_dev, off_dev, info_dev are DEVICE pointers owned
 *    by the caller; the library never frees or retains them.  fm_coeffs arrays
 *    are HOST pointers, read during the call only.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are stream-ordered and asynchronous: the return status reports
 *    argument, configuration and launch errors only.  Per-matrix numerical
 *    status goes to info (device int per matrix, or the optional info_host of the
 *    single-matrix calls after a synchronize):
 *        0       success
 *        > 0     exactly zero pivot: (term index i) * d + (1-based column);
 *                a system that serves two terms (a pair of nodes +c, -c
 *                of the roundoff form, I - c^2 B^2, or a conjugate pair)
 *                reports the index of its first term
 *        -1      FM_FP32_IR: iterative refinement did not reach opts.ir_tol;
 *                FM_BF16_IR: the correction iteration did not converge
 *        -2      non-finite entry in A (or V, or t)
 *        -3      adjoint: nsteps_dev[b] < 1 or > opts.nsteps (not computed)
 *        -4      batched calls: d_dev[b] outside [1, dmax] (matrix b is left
 *                out; its outputs are not written)
 *        -5      fm_rfun: ||tA||_1 > theta, outside the accuracy range of the
 *                set (the result is still computed)
 *        -7      a bounded wait inside a tensor-core kernel or at a grid-wide
 *                barrier of the team path ran out (the kernel stopped early;
 *                the results of the call are invalid)
 *  - Outputs must not alias inputs.
 *  - Scratch: opts.workspace (device, opts.workspace_bytes >= fm_workspace_size)
 *    or, when NULL, a buffer the library keeps per (device, stream): calls on
 *    one stream share it in stream order, calls on different streams use
 *    different buffers and may overlap.  A buffer is taken with
 *    cudaMallocAsync on the call's stream the first time a problem does not
 *    fit it (the smaller one is released with cudaFreeAsync on that stream,
 *    after the work queued before it), so make the first call of each size
 *    before capturing the stream into a graph.  Host threads that share a
 *    stream take turns (a lock per buffer, held until the call has queued
 *    its work).  Buffers are released at process exit; streams are told apart
 *    by handle (cudaStreamPerThread by calling thread).  A caller-provided
 *    opts.workspace must not be used by two calls that overlap on the GPU.
 *  - Errors: FM_EINVAL (bad pointer, value or coefficient set), FM_ESHAPE (bad
 *    dimension or leading dimension, or d beyond what the kernels support),
 *    FM_ENOMEM, FM_ECUDA (launch or runtime failure).  fm_last_error() returns
 *    a message for the calling thread's last failure.
 */
#ifndef FM_H_
#define FM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FM_OK = 0,
  FM_EINVAL = 1,
  FM_ESHAPE = 2,
  FM_ENOMEM = 3,
  FM_ECUDA = 4,
  FM_ESINGULAR = 5,
  FM_ENOCONV = 6,
  FM_ETIMEOUT = 7
} fm_status;

/* A coefficient set (Sec. 2 and 4).  k terms with nodes c_i and weights b_i
 * (c_i = 0 terms allowed: they cost no solve).  conj_pair = 1 means each term
 * stands for 2 Re(b_i / (1 - c_i x)) with complex c_i, b_i (Eq. Pade4, Pade4phi1):
 * on real matrices every such term is one real system
 * I - 2 Re(c_i) B + |c_i|^2 B^2 after one product B^2 (Sec. 1: one product x^2
 * and one inverse per pair of complex-conjugate roots); on complex matrices
 * (z functions) the term means its analytic form
 * b_i / (1 - c_i x) + conj(b_i) / (1 - conj(c_i) x), two complex systems.
 * The tridiagonal action and the adjoint take sets with conj_pair = 0 only.
 * a0 = r(0); d1, d2 = hybrid polynomial part (Eq. Frac10).
 * order = s of Eq. (approx1); theta = ||B|| threshold for the target tolerance
 * (Sec. 3).  Arrays are host memory of length k; c_im / b_im may be NULL for
 * real sets.  k <= FM_MAX_TERMS. */
#define FM_MAX_TERMS 16
typedef struct {
  int k;
  const double* c_re;
  const double* c_im;
  const double* b_re;
  const double* b_im;
  int conj_pair;
  double a0, d1, d2;
  int order;
  double theta;
} fm_coeffs;

/* Built-in sets.  The b_i are those printed in the paper, or (FM_R8_PHI1,
 * FM_R4_PHI1_A5, FM_R8_COS, FM_R8_SIN, FM_R8_PHI2) the exact solution of
 * Eq. (LinearEqsbi) with the printed c_i and the Taylor coefficients a_k of
 * the function.  theta is computed for the double-precision unit roundoff
 * 2^-53 from the forward bound of Sec. 3. */
enum {
  FM_R4 = 0,         /* Eq. Frac4ci/Frac4bi, alpha = 5, exp, 4 solves          */
  FM_R4_PHI1 = 1,    /* Sec. 4.1, alpha = 6, phi_1, 4 solves                   */
  FM_R4_PHI1_A5 = 2, /* alpha = 5 nodes, phi_1 weights (shares R4's solves)    */
  FM_R8 = 3,         /* Eq. Frac8ci/Frac8bi, alpha = 5, exp, 8 solves           */
  FM_R8_PHI1 = 4,    /* R8 nodes, phi_1 weights (shares R8's solves)            */
  FM_R5 = 5,         /* Eq. Frac5bi0, exp, 5 solves                             */
  FM_R10 = 6,        /* Eq. Frac10ci/Frac10bi, hybrid, 10 solves + B^2          */
  FM_R10_STAR = 7,   /* Eq. Frac10ciNO/Frac10biNO, hybrid, 10 solves + B^2      */
  FM_PADE22 = 8,     /* Eq. Pade4, one conjugate pair                           */
  FM_PADE22_PHI1 = 9,/* Eq. Pade4phi1, one conjugate pair                       */
  FM_R8_COS = 10,    /* R8 nodes, cos weights (Sec. 1, with fm_cossin)          */
  FM_R8_SIN = 11,    /* R8 nodes, sin weights (shares R8_COS's solves)          */
  FM_R8_PHI2 = 12,   /* R8 nodes, phi_2 weights (Sec. 1, the phi-functions)     */
  FM_FRAC4_EXP = 13, /* c_i = 1/(i+1), i = 1..5, Eq. Frac4bi0 (exp)             */
  FM_FRAC4_PHI1 = 14,/* same nodes, the printed phi_1 weights                   */
  FM_FRAC4_LOG1M = 15/* same nodes, the printed log(1 - x) weights (fm_rfun)    */
};
#define FM_NUM_BUILTIN 16

/* Target functions of a set (its Taylor coefficients a_k, Eq. fB). */
enum { FM_FUNC_EXP = 0, FM_FUNC_PHI1 = 1, FM_FUNC_PHI2 = 2, FM_FUNC_COS = 3, FM_FUNC_SIN = 4,
       FM_FUNC_LOG1M = 5 };

/* Fill *out with built-in set id.  The arrays point to static storage that
 * stays valid for the life of the process.  Returns FM_EINVAL for a bad id. */
fm_status fm_coeffs_builtin(int id, fm_coeffs* out);

/* Forward bound eps(x) = sum_{k>order} |a_k - alpha_k| x^k (Sec. 3) of a set
 * against target function func (FM_FUNC_*), and the x at which it reaches
 * tol.  Host computation in extended precision.  Returns FM_EINVAL on bad
 * arguments. */
fm_status fm_theta(const fm_coeffs* cs, int func, double tol, double* theta_out);

/* Arithmetic of a call (opts.precision).  Every value is accurate to double.
 *  FM_FP64     every step in double on the FP64 pipe (any path).
 *  FM_FP32_IR  one-CTA kernels only: each shifted matrix factored and solved
 *              in single precision, then opts.max_ir_iters steps of iterative
 *              refinement whose residuals are accurate to double (real
 *              matrices: products as exact BF16 digit products on the tensor
 *              cores; complex: double products); info = -1 when the last
 *              correction exceeds opts.ir_tol.
 *  FM_BF16_IR  grid paths only: every matrix product is a BF16 digit product
 *              on the tensor cores with exact accumulation (accurate to
 *              double), and each shifted system is solved by the correction
 *              iteration of FM_PATH_GRID, run to its own stop rule (at most 40
 *              steps; info = -1 if it does not converge); opts.max_ir_iters
 *              and opts.ir_tol are not used.
 *  FM_MIXED    FM_FP32_IR on the one-CTA kernels, FM_BF16_IR on the grid
 *              paths, double on the team path (the default). */
enum { FM_FP64 = 0, FM_FP32_IR = 1, FM_BF16_IR = 2, FM_MIXED = 3 };
enum { FM_ROUNDOFF = 0, FM_PLAIN = 1 }; /* Eq. ParallRoundOff or Eq. rat1       */
/* Execution path.  FM_PATH_CTA: one thread block per matrix, every step in it
 * (LU with partial pivoting of each shifted matrix; d <= fm_max_dim()).
 * FM_PATH_GRID: every step is one launch over the whole GPU -- one matrix of
 * any order (single-matrix calls), or a whole batch (batched exp, phi_1 and
 * phi_1 V, dmax <= fm_max_dim()); each shifted system (I - c_i B) Y_i = c_i B is solved
 * by the residual-correction (Newton-Schulz) iteration
 * Y <- Y + (I + Y)(C - (I - C) Y), C = c_i B, whose only heavy steps are matrix
 * products, until the largest residual entry times d is below 2^-30 (then one
 * more correction); it needs the spectral radius of c_i B well below 1, as
 * every set here gives with ||B||_1 <= theta (||c_i B||_1 <= 0.05).  Products
 * run on the FP64 pipe (FM_FP64) or as BF16 digit products on the tensor cores
 * with exact accumulation (FM_BF16_IR, FM_MIXED), both accurate to double.
 * The action forms the matrix r(B) once and applies it N times.  Calls on
 * this path synchronize their stream (s or N, the batch orders and the
 * iteration counts are read on the host).
 * FM_PATH_TEAM: single-matrix exp (fm_expm, fm_zexpm, fm_rfun) of order
 * d <= 512 in double (FM_FP64 or FM_MIXED): one cooperative launch whose thread
 * blocks share every step -- the shifted systems are factored on separate
 * blocks at once (Sec. 2: one processor per system), their d right-hand-side
 * columns solved in column blocks across the grid, and B^2 and each squaring
 * computed as 8 x 8 output tiles over all blocks; grid-wide barriers (bounded
 * waits: info -7 when one runs out) separate the steps.  The call
 * synchronizes its stream only to read a status that was asked for.
 * FM_PATH_AUTO: FM_BF16_IR calls, single-matrix calls with d > fm_max_dim(),
 * and batched exp, phi_1, phi_1 V and cos/sin in FM_MIXED with dmax >= 64 take
 * the grid path; single-matrix exp with d <= 512 in FM_FP64 or FM_MIXED the
 * team path; everything else the one-CTA kernels.  After fm_autotune (or
 * with its FM_TUNE_CACHE), batched matrix functions in FM_MIXED are split at
 * the measured order d* instead.  A precision value and a path
 * that do not go together (FM_FP32_IR with FM_PATH_GRID, FM_BF16_IR with
 * FM_PATH_CTA, a batched action on the grid path) give FM_EINVAL. */
enum { FM_PATH_AUTO = 0, FM_PATH_CTA = 1, FM_PATH_GRID = 2, FM_PATH_TEAM = 3 };

typedef struct {
  int precision;      /* FM_FP64, FM_FP32_IR, FM_BF16_IR or FM_MIXED (above)    */
  int form;           /* FM_ROUNDOFF (default) or FM_PLAIN                      */
  int max_ir_iters;   /* refinement steps for FM_FP32_IR (default 2)            */
  double ir_tol;      /* info = -1 when the last correction exceeds ir_tol times
                         the solution (max norms); 0 disables (default 1e-8)    */
  double anorm;       /* > 0: use anorm*|t| in place of ||tA||_1 to pick s / N  */
  int s_fixed;        /* >= 0: force s for matrix functions (default -1); -2:
                         s = 0 and info -5 when ||tA||_1 > theta (fm_rfun)     */
  long nsteps;        /* > 0: force N for actions (default 0)                   */
  void* workspace;    /* device scratch or NULL                                 */
  size_t workspace_bytes;
  int path;           /* FM_PATH_AUTO (default), _CTA, _GRID or _TEAM            */
} fm_opts;

/* Defaults: FM_MIXED, FM_ROUNDOFF, 2 refinement steps, ir_tol 1e-8, automatic
 * s and N, library-managed workspace, FM_PATH_AUTO. */
void fm_opts_default(fm_opts* o);

/* Job kinds for fm_workspace_size. */
enum { FM_JOB_EXPM = 0, FM_JOB_PHI1 = 1, FM_JOB_EXPMV = 2, FM_JOB_PHI1MV = 3,
       FM_JOB_ZEXPM = 4, FM_JOB_ZEXPMV = 5, FM_JOB_EXPMV_ADJ = 6, FM_JOB_COSSIN = 7,
       FM_JOB_RFUN = 8 };

/* Bytes of device scratch a call of that job needs for matrices up to dmax, m
 * vectors, k terms, on the current device. */
size_t fm_workspace_size(int job, int batch, int dmax, int m, int k, const fm_opts* opts);

/* Largest d of the one-CTA-per-matrix kernels: every batched call, and the
 * single-matrix calls on FM_PATH_CTA.  Single-matrix exp / phi_1 and their
 * actions (real and complex) of larger order take the grid path, limited by
 * device memory only (fm_workspace_size with batch = 1). */
int fm_max_dim(void);

/* ---- single matrix ------------------------------------------------------ */

/* F = exp(tA) ~ r(B)^(2^s), B = tA/2^s (Sec. 1, Eq. ParallRoundOff).
 * A: d x d (lda), F: d x d (ldf).  info_host (nullable, host): per-matrix status,
 * valid after the stream is synchronized; s_host (nullable, host): chosen s. */
fm_status fm_expm(const fm_coeffs* cs, int d, const double* A, int lda, double t, double* F,
                  int ldf, const fm_opts* opts, void* stream, int* info_host, int* s_host);

/* Phi = phi_1(tA) and (if E != NULL) E = exp(tA), both from the same resolvents
 * (Sec. 2: one set of solves, two sets of weights), then s doublings
 * (Phi, E) <- ((E + I) Phi / 2, E^2) (Sec. 1).  theta = min of the two sets. */
fm_status fm_phi1(const fm_coeffs* ce, const fm_coeffs* cphi, int d, const double* A, int lda,
                  double t, double* Phi, int ldp, double* E, int lde, const fm_opts* opts,
                  void* stream, int* info_host, int* s_host);

/* W = exp(tA) V by N steps W <- r(B) W, B = tA/N, with one factorization per
 * term reused by all steps and all m columns (Sec. 1, 2; Eq. Frac10R: one
 * product B W per step).  V, W: d x m (ldv, ldw). */
fm_status fm_expmv(const fm_coeffs* cs, int d, const double* A, int lda, double t, int m,
                   const double* V, int ldv, double* W, int ldw, const fm_opts* opts,
                   void* stream, int* info_host, long* nsteps_host);

/* W = phi_1(tA) V: phi_1(tA) by fm_phi1's doubling, then one product. */
fm_status fm_phi1mv(const fm_coeffs* ce, const fm_coeffs* cphi, int d, const double* A, int lda,
                    double t, int m, const double* V, int ldv, double* W, int ldw,
                    const fm_opts* opts, void* stream, int* info_host, int* s_host);

/* Complex variants: A, V, F, W interleaved complex double; c_i, b_i complex
 * (conj_pair must be 0). */
fm_status fm_zexpm(const fm_coeffs* cs, int d, const double* A, int lda, double t, double* F,
                   int ldf, const fm_opts* opts, void* stream, int* info_host, int* s_host);
fm_status fm_zexpmv(const fm_coeffs* cs, int d, const double* A, int lda, double t, int m,
                    const double* V, int ldv, double* W, int ldw, const fm_opts* opts,
                    void* stream, int* info_host, long* nsteps_host);

/* ---- batches of independent matrices (one launch) ------------------------ */
/* Matrix b has order d_dev[b] <= dmax and is stored densely (leading dimension
 * d_dev[b]) at A + off_dev[b] (elements; complex: complex elements); its result
 * goes to the same offset of F (or Phi/E/W; for actions V and W use voff_dev
 * with leading dimension m).  t_dev[b] is its time.  info_dev[b] receives its
 * status and s_dev[b] (nullable) its s or N.  Work is ordered largest d first
 * and spread over persistent CTAs, one matrix per CTA at a time. */
fm_status fm_expm_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                          const int64_t* off_dev, const double* A, const double* t_dev,
                          double* F, int* info_dev, int* s_dev, const fm_opts* opts,
                          void* stream);
fm_status fm_phi1_batched(const fm_coeffs* ce, const fm_coeffs* cphi, int batch, int dmax,
                          const int* d_dev, const int64_t* off_dev, const double* A,
                          const double* t_dev, double* Phi, double* E, int* info_dev,
                          int* s_dev, const fm_opts* opts, void* stream);
fm_status fm_expmv_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                           const int64_t* off_dev, const double* A, const double* t_dev, int m,
                           const int64_t* voff_dev, const double* V, double* W, int* info_dev,
                           int* s_dev, const fm_opts* opts, void* stream);
fm_status fm_phi1mv_batched(const fm_coeffs* ce, const fm_coeffs* cphi, int batch, int dmax,
                            const int* d_dev, const int64_t* off_dev, const double* A,
                            const double* t_dev, int m, const int64_t* voff_dev,
                            const double* V, double* W, int* info_dev, int* s_dev,
                            const fm_opts* opts, void* stream);
fm_status fm_zexpm_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                           const int64_t* off_dev, const double* A, const double* t_dev,
                           double* F, int* info_dev, int* s_dev, const fm_opts* opts,
                           void* stream);
fm_status fm_zexpmv_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                            const int64_t* off_dev, const double* A, const double* t_dev, int m,
                            const int64_t* voff_dev, const double* V, double* W, int* info_dev,
                            int* s_dev, const fm_opts* opts, void* stream);

/* ---- other functions from the same resolvents (Sec. 1, Sec. 2) ---------- */
/* C = cos(tA) and (if S != NULL) S = sin(tA), real A: both from one set of
 * shifted solves with two weight vectors cc and cs over the same nodes
 * (Sec. 2; FM_R8_COS and FM_R8_SIN), B = tA/2^s with theta the smaller of the
 * two sets', then s steps of the double-angle formulae of Sec. 1,
 * (C, S) <- (2 C^2 - I, 2 S C).  Each step can multiply the rounding by about
 * 4 ||C||: the results are accurate to about 4^s u.  Layout, paths and status
 * as fm_phi1 (C takes the place of Phi, S of E). */
fm_status fm_cossin(const fm_coeffs* cc, const fm_coeffs* cs, int d, const double* A, int lda,
                    double t, double* C, int ldc, double* S, int lds, const fm_opts* opts,
                    void* stream, int* info_host, int* s_host);
fm_status fm_cossin_batched(const fm_coeffs* cc, const fm_coeffs* cs, int batch, int dmax,
                            const int* d_dev, const int64_t* off_dev, const double* A,
                            const double* t_dev, double* C, double* S, int* info_dev, int* s_dev,
                            const fm_opts* opts, void* stream);

/* F = r(tA) for any set, with no range reduction: B = tA, F = r(B) (Sec. 2:
 * f(B) ~ r(B) for sufficiently small ||B||).  For functions the paper gives no
 * scaling for, such as log(1 - x) with the weights printed after Eq.
 * Frac4bi0 (FM_FRAC4_LOG1M), or phi_2 (FM_R8_PHI2).  info = -5 when
 * ||tA||_1 > theta (the result is still written).  Paths, layout and the other
 * status values as fm_expm; opts.s_fixed is ignored. */
fm_status fm_rfun(const fm_coeffs* cs, int d, const double* A, int lda, double t, double* F,
                  int ldf, const fm_opts* opts, void* stream, int* info_host);
fm_status fm_rfun_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                          const int64_t* off_dev, const double* A, const double* t_dev, double* F,
                          int* info_dev, const fm_opts* opts, void* stream);

/* ---- adjoint of the action (real, roundoff form, one vector) ----------- */
/* For each matrix of the batch: the forward map w_0 = v, w_q = r(B) w_{q-1}
 * (q = 1..N, B = tA/N with N = nsteps_dev[b] fixed, as fm_expmv computes it),
 * and given wbar = dL/dw_N, the gradients Abar = dL/dA (d x d at off_dev[b]) and
 * vbar = dL/dv (d at voff_dev[b]).  The reverse sweep reuses the forward
 * factorizations: lambda = M_i^{-T} (b_i wbar_q), Bbar += c_i lambda Y_iq^T,
 * ubar = sum c_i lambda, Bbar += ubar w_{q-1}^T, wbar_{q-1} = a0 wbar_q + B^T ubar.
 * W receives w_N.  Always double precision. */
fm_status fm_expmv_adjoint_batched(const fm_coeffs* cs, int batch, int dmax, const int* d_dev,
                                   const int64_t* off_dev, const double* A, const double* t_dev,
                                   const long* nsteps_dev, const int64_t* voff_dev,
                                   const double* v, const double* wbar, double* W,
                                   double* Abar, double* vbar, int* info_dev,
                                   const fm_opts* opts, void* stream);

/* ---- step a1 alone: the scaling each call would choose ------------------ */
/* For each matrix of a batch (layout of the batched calls: order d_dev[b] <=
 * dmax, dense at A + off_dev[b], time t_dev[b]): eta = ||t_b A_b||_1, the
 * largest column sum of |t_b a_ij| (or opts.anorm |t_b|), and then what the
 * call of that job chooses from it (Sec. 1: N such that ||A/N|| < theta, N = 2^s
 * for scaling and squaring; theta from the forward bound of Sec. 3):
 *   job FM_JOB_EXPM, FM_JOB_PHI1, FM_JOB_PHI1MV, FM_JOB_ZEXPM:
 *       out_dev[b] = s, the smallest s >= 0 with eta / 2^s <= theta
 *       (opts.s_fixed >= 0: s_fixed);
 *   job FM_JOB_EXPMV, FM_JOB_ZEXPMV, FM_JOB_EXPMV_ADJ:
 *       out_dev[b] = N = max(1, ceil(eta / theta)) (opts.nsteps > 0: nsteps),
 *       the step count that fm_expmv_adjoint_batched takes as nsteps_dev.
 * theta is that of cs (phi_1 jobs: the smaller of cs and cphi).  FM_JOB_Z*
 * read A as complex.  out_dev (device, 64-bit long per matrix), info_dev
 * (device): 0, -2 (non-finite entry of A_b or t_b) or -4 (d_dev[b] outside
 * [1, dmax]; out_dev[b] = 0).  One launch, no synchronization.  Errors:
 * FM_EINVAL (NULL pointer, bad job or set), FM_ESHAPE, FM_ECUDA. */
fm_status fm_select_batched(const fm_coeffs* cs, const fm_coeffs* cphi, int job, int batch,
                            int dmax, const int* d_dev, const int64_t* off_dev, const double* A,
                            const double* t_dev, long* out_dev, int* info_dev, const fm_opts* opts,
                            void* stream);

/* ---- actions of tridiagonal matrices (Sec. 2.1, Sec. 5) ------------------ */
/* W_b = r(B_b)^(N_b) V_b ~ exp(t_b A_b) V_b for a batch of tridiagonal A_b of one
 * order d: the action recurrence of Sec. 1 with B_b = (t_b / N_b) A_b and
 * N_b = max(1, ceil(||t_b A_b||_1 / theta)) (opts.anorm > 0: anorm |t_b| in place
 * of the norm; opts.nsteps > 0: N_b = nsteps).  Each shifted matrix I - c_i B_b
 * is tridiagonal (Sec. 2.1): it is factored once per call by the Thomas
 * algorithm, without pivoting, and every step solves it in 8d flops (plain
 * form, Eq. rat1, the paper's R_10) or, with the product B v, 13d (roundoff
 * form, Eq. ParallRoundOff, the paper's R'_10).  Same N and the same rational
 * function as fm_expmv on the dense matrix.
 *
 * Layout (all DEVICE, double, batch-interleaved): element k of system b is at
 * k * batch + b in dl (sub-diagonal A[k][k-1], k >= 1; the k = 0 slot is not
 * read), dd (diagonal A[k][k]), du (super-diagonal A[k][k+1], k <= d - 2; the
 * k = d - 1 slot is not read), V and W.  t_dev[b]: time of system b.
 * info_dev[b]: 0; -2 for a non-finite entry of A_b, V_b or t_b (W_b is not
 * written); or (term index i) * d + (1-based row) for an exactly zero pivot of
 * the first such I - c_i B_b (W_b is not written).  nsteps_dev[b] (nullable):
 * N_b.  dl and du may be NULL when d = 1.  Double precision whatever
 * opts.precision says; the coefficient set must have real nodes, at least one
 * of them nonzero, and one function (no phi_1 weights).  Scratch:
 * fm_trid_workspace_size bytes in opts.workspace, or the library's buffer.
 * Stream-ordered, no host synchronization.  Errors: FM_EINVAL (NULL pointer,
 * complex or empty node set), FM_ESHAPE (batch or d < 1), FM_ENOMEM, FM_ECUDA. */
fm_status fm_trid_expmv_batched(const fm_coeffs* cs, int batch, int d, const double* dl,
                                const double* dd, const double* du, const double* t_dev,
                                const double* V, double* W, int* info_dev, int* nsteps_dev,
                                const fm_opts* opts, void* stream);

/* Bytes of device scratch of fm_trid_expmv_batched for batch systems of order
 * d and a set of k terms (0 for a bad argument). */
size_t fm_trid_workspace_size(int batch, int d, int k);

/* ---- autotuner: which kernels take which orders of a batch -------------- */
/* The paper has no counterpart (it has no hardware): this measures, on the
 * current device, batches of matrix functions (job FM_JOB_EXPM, FM_JOB_PHI1 or
 * FM_JOB_COSSIN with sets ce, cp) of each probe order d in {16, 32, 48, 64, 96,
 * 128, ..., 1024} up to dmax, on the one-CTA kernels (FM_FP32_IR) and on the
 * batched grid path (FM_BF16_IR): synthetic matrices with ||A||_1 about 4,
 * the best of two calls timed with CUDA events on the stream.  It records d*,
 * the smallest probe order from which the grid path is at least as fast at
 * every larger probe (1: the grid path everywhere; dmax + 1: nowhere).  From
 * then on, batched calls of that job in FM_MIXED with FM_PATH_AUTO on this
 * device run the orders below d* on the one-CTA kernels and the rest on the
 * grid path (two launches one after the other; each leaves the other's
 * matrices and status alone).  If the environment variable FM_TUNE_CACHE
 * names a file, the result is appended to it as "device|job|d*" and read back
 * by the first batched call of a later process.  table_out (nullable, host,
 * 3 x 16 doubles): per probe (d, microseconds per matrix on the one-CTA
 * kernels, on the grid path); nprobe_out: the number of probes.  Allocates its
 * probe batches (cudaMallocAsync) and synchronizes the stream.  Errors:
 * FM_EINVAL (job, sets), FM_ESHAPE (dmax), FM_ECUDA, FM_ENOMEM. */
fm_status fm_autotune(const fm_coeffs* ce, const fm_coeffs* cp, int job, int dmax,
                      const fm_opts* opts, void* stream, int* dstar_out, double* table_out,
                      int* nprobe_out);

/* Forget every tuned d* of this process: FM_PATH_AUTO takes the fixed rule
 * again, unless FM_TUNE_CACHE (read again by the next batched call) names a
 * file with entries for this device. */
void fm_autotune_reset(void);

/* ---- actions of banded matrices (Sec. 1, Sec. 5.1) ----------------------- */
/* W_b = r(B_b)^(N_b) V_b ~ exp(t_b A_b) V_b for a batch of banded A_b of one
 * order d and half bandwidth p (1: tridiagonal, 2: pentadiagonal): the
 * action recurrence of Sec. 1 as in fm_trid_expmv_batched.  Every shifted
 * matrix I - c_i B_b is banded with the same p (Sec. 1: a pentadiagonal system
 * is solved in 15d flops and the product A v costs 9d), factored once per call
 * by banded LU without pivoting (|c_i| ||B||_1 is far below 1/2 at
 * ||B||_1 <= theta: diagonally dominant) and solved in every step.  p = 1 runs
 * fm_trid_expmv_batched on the same layout.
 *
 * Layout (DEVICE, double, batch-interleaved): diagonal j = 0 .. 2p (offset
 * o = j - p) holds A[k][k + o] of system b at (j d + k) batch + b; entries
 * with k + o outside [0, d) are not read.  V, W, t_dev, info_dev, nsteps_dev and
 * the status values as fm_trid_expmv_batched (info: 0, -2 non-finite entry,
 * or i d + row for an exactly zero pivot of term i).  Double precision; the set
 * must have real nodes (conj_pair = 0), at least one nonzero, and one function.
 * Scratch: fm_band_workspace_size bytes.  Stream-ordered, no host
 * synchronization.  Errors: FM_EINVAL (NULL pointer, p not 1 or 2, bad set),
 * FM_ESHAPE (batch or d < 1), FM_ENOMEM, FM_ECUDA. */
fm_status fm_band_expmv_batched(const fm_coeffs* cs, int batch, int d, int p,
                                const double* diags, const double* t_dev, const double* V,
                                double* W, int* info_dev, int* nsteps_dev, const fm_opts* opts,
                                void* stream);

/* Bytes of device scratch of fm_band_expmv_batched (0 for a bad argument). */
size_t fm_band_workspace_size(int batch, int d, int p, int k);

/* ---- exp(tA) without any device allocation ------------------------------ */
/* The paper has no counterpart: this is a deployment variant of fm_expm for
 * callers that cannot allocate device memory (code that runs where cudaMalloc
 * is forbidden or could deadlock, such as a custom allocator or a memory-pool
 * hook, and hosts that own every device byte).  Same arguments and results as
 * fm_expm on the one-CTA kernel (real, one matrix), but its scratch is a fixed
 * array inside the library image; opts.workspace is ignored.
 *   - d <= FM_NOALLOC_MAX_DIM and the scratch the call needs must fit in
 *     FM_NOALLOC_SCRATCH_BYTES, else FM_ESHAPE with a message.
 *   - opts.path = FM_PATH_GRID or FM_PATH_TEAM and opts.precision =
 *     FM_BF16_IR are rejected (FM_EINVAL): those paths need their own scratch.
 *     (fm_expm itself takes the team path for d <= 512 by default; the
 *     results agree to the double-accurate bar.)
 *   - Every call uses the same array: calls that overlap on the GPU (several
 *     streams or host threads) race and give wrong results; serialize them.
 *   - CUDA loads the library's device code, the array included, on a device
 *     when it is first used there: the first call on each device commits the
 *     array and looks up its device address with that device current, and can
 *     fail with FM_ECUDA when the device is out of memory.  Make that first call
 *     once per device as a warm-up, before any stream capture and outside any
 *     code that must not allocate; later calls allocate nothing.
 *   - Not for host functions enqueued on a stream (cudaLaunchHostFunc): CUDA
 *     allows no CUDA call there, and this entry point launches kernels.
 *   - info_host / s_host (nullable) make the call synchronize the stream. */
#define FM_NOALLOC_MAX_DIM 128
#define FM_NOALLOC_SCRATCH_BYTES (2u << 20)
fm_status fm_expm_noalloc(const fm_coeffs* cs, int d, const double* A, int lda, double t,
                          double* F, int ldf, const fm_opts* opts, void* stream, int* info_host,
                          int* s_host);

/* Message for the calling thread's last failing call ("" if none). */
const char* fm_last_error(void);

/* Work done by the calling thread's last call on the grid path (zeros after a
 * call on the one-CTA path): matrix products, their algorithmic flops (2MNK
 * real, 8MNK complex), the tensor-core flops of their digit products (the
 * digit pairs kept, 28 at full accuracy, per product flop; 0 on the FP64
 * pipe), and the largest
 * number of correction steps one shifted system took, the number of kernel
 * launches of the call, and the summed CUDA-event time of its tensor-core tile
 * launches (events recorded on the call's stream around each).  The library has no
 * counterpart in the paper; it serves measurement. */
typedef struct {
  long long products;
  double product_flops;
  double digit_flops;
  int corrections;
  long long launches;  /* kernels the call launched */
  double tile_ms;      /* CUDA-event time of the tensor-core tile launches */
} fm_stats;
void fm_last_stats(fm_stats* out);

/* Library version string. */
const char* fm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FM_H_ */
