/*
 * fst.h -- C ABI of the GB300 fast Slepian projection library (libfst_gb300.so).
 *
 * The library computes the fast approximation of S_K S_K^* y of Corollary 2 and
 * Section 1.3 ("Fast projections onto the range of S_K") of Karnik, Zhu, Wakin,
 * Romberg, Davenport, "The Fast Slepian Transform" (arXiv:1611.04950):
 *
 *     P_fast y = B_{N,W} y + S_T (D o (S_T^T y)),
 *
 * where B_{N,W} is the prolate matrix (Eq. "Prolate matrix", Section 1.2) applied as
 * a zero-padded length-M FFT convolution (M = smallest power of two >= 2N,
 * Section 4.1), S_T holds the Slepian basis vectors whose eigenvalues lie in the
 * transition band, and D = 1[l<K] - lambda_l (the U1 U2^* factors of the proof of
 * Corollary 2).  The same machinery gives the truncated pseudoinverse of B
 * (Corollary 3, D = 1/lambda - lambda on l<K, -lambda on l>=K) and the Tikhonov
 * operator (Corollary 4, B/(1+alpha) + U5 U5^*).
 *
 * Conventions for every entry point:
 *   - Status codes are returned; the library never aborts.  fst_last_error() gives
 *     a message for the last failing call on the calling host thread.
 *   - Device pointers are caller-owned CUDA device memory; the library never frees
 *     them.  Host pointers are plain host memory (pinned memory copies faster).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All device
 *     work of a call is enqueued on it; calls return before the work completes
 *     unless stated otherwise.
 *   - Signals are stored one after another: signal b starts at element b*ld
 *     (ld >= N; ld = 0 means ld = N).  Real dtypes hold N reals per signal,
 *     complex dtypes N interleaved (re, im) pairs.
 *   - A plan is not thread-safe: calls on one plan must be serialised by the caller
 *     (they share the plan's device workspace).
 */
#ifndef FST_GB300_H
#define FST_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fst_plan_s *fst_plan_t;

typedef enum {
  FST_OK = 0,
  FST_EINVAL = 1,          /* an argument is out of range                       */
  FST_ENOMEM = 2,          /* device or host allocation failed                  */
  FST_ECUDA = 3,           /* a CUDA runtime call or kernel launch failed       */
  FST_ENOCONVERGE = 4,     /* plan-time eigen-solver did not converge           */
  FST_ETIMEOUT = 5,        /* a bounded device wait gave up                     */
  FST_EUNSUPPORTED = 6     /* valid request this build does not handle          */
} fst_status;

typedef enum {
  FST_F32 = 0,   /* real float32        */
  FST_F64 = 1,   /* real float64        */
  FST_C64 = 2,   /* complex float32 (interleaved re, im) */
  FST_C128 = 3   /* complex float64 (interleaved re, im) */
} fst_dtype;

typedef enum {
  FST_OP_PROJECT = 0,   /* S_K S_K^*                   (Corollary 2) */
  FST_OP_PINV = 1,      /* rank-K truncated B^dagger   (Corollary 3) */
  FST_OP_TIKHONOV = 2   /* (B^2 + alpha I)^{-1} B      (Corollary 4) */
} fst_op;

/*
 * fst_plan -- precomputation of Section 1.3 (last paragraph) and Section 4.1.
 * Computes, on the GPU in FP64, the Slepian basis vectors of the eigen-window
 * around K (bisection on Slepian's commuting tridiagonal matrix, split by parity,
 * then inverse iteration), their eigenvalues lambda_l = s_l^T B s_l (FP64 FFT
 * convolution), the transition set T = {l : |1[l<K] - lambda_l| > eps}, D, the
 * real sinc spectrum DFT_M(c) (FP64, stored FP32 and FP64) and the twiddle tables.
 *   out     receives the new plan (owned by the library; free with fst_destroy).
 *   N       signal length, 1 <= N <= 2^23.
 *   W       half-bandwidth, 0 < W < 1/2.
 *   K       number of Slepian vectors kept, 0 <= K <= N; K < 0 selects
 *           round(2NW) with halves rounded away from zero (Section 4.1).
 *   eps     tolerance, 0 < eps < 1/2 (Theorem 1, Corollary 2).
 *   stream  stream for the plan-time kernels; the call synchronises it.
 * K need not satisfy the band condition of Corollary 2; T then grows.
 * Cost: the Sturm counts and the tridiagonal LU are serial over the N/2 entries of
 * a reduced matrix, in FP64 (both parities of the window in one batch of targets);
 * on a GB300 about 0.16 s at N = 65536, 2.6 s at N = 2^20 and 10-13 s at N = 2^22.
 * Errors: FST_EINVAL, FST_ENOMEM, FST_ECUDA, FST_ENOCONVERGE.
 */
fst_status fst_plan(fst_plan_t *out, int64_t N, double W, int64_t K, double eps,
                    void *stream);

/*
 * fst_plan_op -- as fst_plan, for the operator `op` (fst_op).  alpha is the
 * Tikhonov parameter (> 0, FST_OP_TIKHONOV only; ignored otherwise).  For
 * Tikhonov the transition set is {alpha(1+alpha)eps < lambda < 1 - eps/3}
 * (Corollary 4) and the Toeplitz part is scaled by 1/(1+alpha).
 */
fst_status fst_plan_op(fst_plan_t *out, int64_t N, double W, int64_t K, double eps,
                       int op, double alpha, void *stream);

/*
 * fst_plan_info -- sizes of a plan.  Any output pointer may be NULL.
 *   K, r (= |T|), M (FFT length), window_lo / window_hi (eigen-window searched,
 *   inclusive descending-lambda indices).
 */
fst_status fst_plan_info(fst_plan_t plan, int64_t *K, int64_t *r, int64_t *M,
                         int64_t *window_lo, int64_t *window_hi);

/*
 * fst_plan_export -- copies the plan's transition data to HOST arrays (any may be
 * NULL): idx[r] (int64 indices l in T, ascending), lam[r] (lambda_l, FP64),
 * D[r] (FP64), S_T[N*r] (FP64, column j = s^(idx[j]) contiguous, unit norm).
 * Synchronous.
 */
fst_status fst_plan_export(fst_plan_t plan, int64_t *idx, double *lam, double *D,
                           double *S_T);

/*
 * fst_project -- P_fast y for `batch` signals resident on the device
 * (Section 1.3, "Fast projections onto the range of S_K").
 *   y, out  device pointers, `batch` signals each, stride ld (0 = N).  y and out
 *           may be equal (in place); otherwise they must not overlap.
 *   dtype   FST_F32 / FST_C64: FP32 FFT convolution and FP32-accurate correction;
 *           FST_F64 / FST_C128: the same kernels in FP64.
 * Real signals are processed two at a time as the real and imaginary parts of
 * one complex FFT (B and S_T are real, so they do not mix).
 * FP32: when y is 16-byte aligned, its row stride is a multiple of 16 bytes and the
 * batch has more than 32 signal rows (real signals, or two per complex signal),
 * S_T^T y for the whole batch runs on the tensor cores (TF32 with a hi/lo split,
 * three products); smaller batches use FP32 CUDA-core sums, other layouts mma.sync
 * kernels -- other summation orders, same accuracy.  Results are bit-for-bit
 * repeatable for the same call.
 * Errors: FST_EINVAL (NULL pointer, batch < 0, ld < N), FST_ENOMEM, FST_ECUDA,
 * FST_ETIMEOUT (see below).
 * Device waits: every wait of the tensor-core kernel on its own copies and products
 * is bounded (2 s of wall time).  Should one run out, that launch stops issuing work,
 * waits (bounded) for what it already issued, frees its tensor memory, writes NaN
 * for the affected outputs and raises the plan's error word.  The call itself is
 * asynchronous and cannot see this; the word is reported as FST_ETIMEOUT by
 * fst_sync(), by fst_project_host() of that call, or by the next fst_project /
 * fst_apply_prolate / fst_project_noalloc / fst_coeffs call on the plan, which then
 * enqueues nothing.  Reporting clears the word.
 * batch == 0 is a no-op returning FST_OK.
 */
fst_status fst_project(fst_plan_t plan, const void *y, void *out, int64_t batch,
                       int64_t ld, int dtype, void *stream);

/*
 * fst_project_host -- as fst_project, with y and out in HOST memory (contiguous,
 * ld = N).  The batch is copied to the device, projected and copied back in
 * chunks on `stream`, overlapping copies with compute (four chunks in flight; the
 * first and last chunks are a quarter of the others); returns after the result is
 * in `out` (synchronous).  Pinned host memory gives the full link bandwidth.  The
 * results are bit-for-bit those of fst_project on the whole batch.  Device scratch:
 * eight chunk buffers of up to FST_HOST_CHUNK_MB (default 64) MiB, allocated on the first
 * call of a thread and kept for its later calls.
 */
fst_status fst_project_host(fst_plan_t plan, const void *y, void *out, int64_t batch,
                            int dtype, void *stream);

/*
 * fst_apply_prolate -- B_{N,W} y alone (no correction): the Toeplitz product of
 * Eq. "Prolate matrix" by the plan's FFT convolution.  Same arguments as
 * fst_project.
 */
fst_status fst_apply_prolate(fst_plan_t plan, const void *y, void *out, int64_t batch,
                             int64_t ld, int dtype, void *stream);

/*
 * fst_coeffs -- the fast coefficient vector c = T2^* y of the fast factorization
 * S_K S_K^* ~ T1 T2^* (Section 1.3, "A fast factorization of S_K S_K^*"), with
 * T2 = [F_{N,W}  L2  U2]: F_{N,W} the 2NW' lowest DFT vectors / sqrt(N)
 * (Eq. PartialFourierMatrix; 2NW' the odd integer nearest 2NW, ties rounded up),
 * L2 the right factor of Theorem 1's construction (Section 2: CF-ADI factor of the
 * Hilbert matrix with the optimal shifts of the appendix, Taylor factors of A1 and
 * B0, phase ramps D_A, D_B) and U2 = [sqrt(|D_l|) s_l] over the transition set.
 * T1 c reproduces S_K S_K^* y within 2 eps ||y|| (Theorem 1 + Corollary 2).
 *   y       device signals as for fst_project (N must be a power of two).
 *   coeffs  device output, batch x K' complex values (complex64 for FST_F32 /
 *           FST_C64 input, complex128 for FST_F64 / FST_C128), signal b at b*K'.
 *           Per signal: F^* y for DFT bins k = -h..h (2h+1 = 2NW'), then the eight
 *           L2 blocks in the order of the proof ((D_A J Z)^*y, (D_A Z)^*y,
 *           (D_A^* J Z)^*y, (D_A^* Z)^*y, C_A V_A^T D_A^*y, C_A V_A^T D_A y,
 *           C_B V_B^T D_B^*y, C_B V_B^T D_B y; V = centred monomials
 *           ((n - (N-1)/2)/N)^i), then U2^* y.
 * The first call builds the construction's tables (host FP64) and allocates.
 * Errors: FST_EINVAL (NULL, batch < 0, ld < N, non-projection plan),
 * FST_EUNSUPPORTED (N not a power of two), FST_ENOMEM, FST_ECUDA.
 */
fst_status fst_coeffs(fst_plan_t plan, const void *y, void *coeffs, int64_t batch, int64_t ld,
                      int dtype, void *stream);

/*
 * fst_expand -- T1 c for `batch` coefficient vectors: the expansion side of the fast
 * factorization S_K S_K^* ~ T1 T2^* (Section 1.3; T1 = [F_{N,W}  L1  U1] with L1 from the
 * constructive proof of Theorem 1, Section 2, and U1 from Corollary 2), so that
 * fst_expand(fst_coeffs(y)) approximates S_K S_K^T y within 2 eps ||y||.
 *   coeffs  device pointer, batch x K' complex (the layout fst_coeffs writes).
 *   out     device pointer, batch x N complex, contiguous (for real signals the
 *           imaginary part is the approximation's residue, of order eps).
 *   dtype   FST_C64 (FP32 kernels) or FST_C128 (FP64 kernels).
 * Uses the plan's workspace (grown on demand).
 * Errors: FST_EINVAL (NULL, batch < 0, real dtype, non-projection plan),
 * FST_EUNSUPPORTED (N not a power of two), FST_ENOMEM, FST_ECUDA.
 */
fst_status fst_expand(fst_plan_t plan, const void *coeffs, void *out, int64_t batch, int dtype,
                      void *stream);

/*
 * fst_coeffs_info -- sizes of the coefficient vector (any pointer may be NULL):
 * K' = 2NW' + r1 + r, nF = 2NW', r1 = 4 r_H + 4 r_A + 2 (2 r_B - 1) and the ranks
 * r_H, r_A, r_B of Section 2.  Builds the construction's tables on first use.
 */
fst_status fst_coeffs_info(fst_plan_t plan, int64_t *Kprime, int64_t *nF, int64_t *r1,
                           int64_t *rH, int64_t *rA, int64_t *rB);

/*
 * fst_adi_shifts -- HOST helper: the r optimal CF-ADI shifts for A = diag(n + 1/2),
 * n < N (appendix, last remarks): p_k = b dn((2k-1)/(2r) K(m), m), b = N - 1/2,
 * m = 1 - (1/(2N-1))^2, computed by the arithmetic-geometric mean.  out[r].
 */
fst_status fst_adi_shifts(int64_t N, int r, double *out);

/*
 * fst_plan_many -- count plans at once (ragged batches: one plan per signal).
 * Same precomputation as fst_plan for each (N[i], W[i], K[i] or round(2NW) when
 * K is NULL or K[i] < 0, eps[i]), projection operator; the bisection and inverse
 * iteration of all plans' eigen-windows run as one batch of independent targets
 * (about 35 s for 4096 plans with N log-uniform in [1000, 262144] on a GB300).
 * out[count] receives the plans (destroy each with fst_destroy).  On error every
 * plan of the call is freed and out[] is NULL.  Synchronous.
 */
fst_status fst_plan_many(fst_plan_t *out, int64_t count, const int64_t *N, const double *W,
                         const int64_t *K, const double *eps, void *stream);

/*
 * fst_project_ragged -- P_fast y_i for a ragged batch: signal i (device pointer
 * y[i], N_i samples of plans[i]) is projected into out[i] with its own plan.
 * Signals whose transform fits one CTA (FP32 N <= 8192, FP64 N <= 4096) go through
 * one launch per FFT length with per-signal descriptors.  Longer FP32 signals run as
 * batches per FFT length through the four-step kernels (real signals two to a complex
 * transform, each with its own spectrum), with the rank-r corrections of all of them in
 * two launches; longer FP64 signals run one four-step call each.  y[i] == out[i] (in
 * place) is allowed.  The first call with a given (plans, y, out, dtype)
 * signature runs directly and allocates; the second records the whole batch in a
 * CUDA graph on a private stream; later calls replay it on `stream` (set
 * FST_GRAPHS=0 in the environment to always launch directly).  Calls with
 * different signatures keep up to four recorded batches.  A recorded batch is
 * dropped when one of its plans is destroyed, and recorded again when a plan's
 * workspace has been reallocated since (a larger fst_project call on it).
 * Errors: FST_EINVAL (NULL pointers, count < 0), FST_ENOMEM, FST_ECUDA.
 */
fst_status fst_project_ragged(const fst_plan_t *plans, const void *const *y, void *const *out,
                              int64_t count, int dtype, void *stream);

/*
 * fst_ragged_tuning -- the launch grouping the autotuner chose for the four-step signals of
 * a ragged batch, for the (plans, y, out, dtype) signature of an earlier fst_project_ragged
 * call: pairs[lg] = transform slots per launch group of the length class with FFT length
 * 2^lg (a slot holds one complex or two real signals; 0 if the batch has no four-step signal
 * of that length), ms[lg] (may be NULL) = the measured
 * device time of that class with the chosen grouping (0 when no timing ran).  Both arrays
 * have 32 entries.  The first call of a signature times groupings of 16 to 256 MiB of
 * intermediate per class and keeps the fastest (FST_AUTOTUNE=0 in the environment: 128 MiB,
 * untimed); the grouping does not change the arithmetic.  Errors: FST_EINVAL (bad
 * arguments, or no call with this signature).
 */
fst_status fst_ragged_tuning(const fst_plan_t *plans, const void *const *y, void *const *out, int64_t count,
                             int dtype, int64_t *pairs, double *ms);

/*
 * fst_sync -- waits for `stream`, then reports the plan's device error word: FST_ETIMEOUT
 * (and clears the word) when a bounded device wait of an earlier call on the plan gave
 * up (its outputs are NaN; see fst_project), FST_OK otherwise.  Errors: FST_EINVAL
 * (NULL plan), FST_ECUDA (the stream failed).
 */
fst_status fst_sync(fst_plan_t plan, void *stream);

/* fst_destroy -- frees the plan and its device memory, and drops the recorded
 * fst_project_ragged batches that use it (after their launches finish).  NULL-safe. */
fst_status fst_destroy(fst_plan_t plan);

/* fst_last_error -- message of the last failing call on this host thread ("" if none). */
const char *fst_last_error(void);

/* fst_version -- library version string. */
const char *fst_version(void);

/*
 * fst_reduced_tridiagonal -- HOST-only helper exposing the plan's parity split of
 * Slepian's tridiagonal matrix (used by the plan's bisection; exported so the
 * split can be checked without a GPU).  parity 0: symmetric vectors, size
 * ceil(N/2); parity 1: antisymmetric vectors, size floor(N/2).  Writes the size to
 * *n, the diagonal to d[0..n) and the off-diagonal to e[0..n-1) (either array may
 * be NULL to query the size).  The l-th largest eigenvalue of the full matrix is
 * the (l div 2)-th largest of the parity-(l mod 2) matrix.
 */
fst_status fst_reduced_tridiagonal(int64_t N, double W, int parity, int64_t *n,
                                   double *d, double *e);

/*
 * fst_project_noalloc -- fst_project that allocates nothing.  The paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc or cudaFree when
 * they project (for example a process whose memory manager owns all device memory
 * after start-up, or a service that must not stall on the allocator mid-request).
 * fst_project allocates its scratch on demand on the plan's first call; this
 * variant instead uses one fixed array of fst_noalloc_scratch_bytes() = 128 MiB
 * compiled into the library (every GPU that loads the library holds it until the
 * process exits).
 *   Arguments, layout and results: as fst_project (device pointers).  The plan
 *   itself must already exist (fst_plan allocates).
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current, and looks it up again when the
 *   device's context has changed (after a device reset); make that first call before
 *   any stream capture.
 *   Sharing: all calls share the one array and it keeps the last call's contents.
 *   Calls whose work overlaps on the GPU (different streams, or several host
 *   threads) race on it: serialise them.  Nothing in it needs clearing.
 *   Errors: as fst_project; FST_EINVAL (message "signal too long for the fixed
 *   scratch buffer") when the scratch of the four-step path does not fit in the
 *   array: one launch group (one to eight pairs of M-point transforms, M the FFT
 *   length) must fit, so FP32 N > 2^22 and FP64 N > 2^21 are always rejected;
 *   beside it, the FP32 tensor-core correction keeps per-pair partial sums
 *   of about 8 (tc_slices + 1) rpad bytes, so large batches are rejected too (N =
 *   65536, r = 22: about 25 KB per pair, beyond roughly 10,000 real signals).  An
 *   emulated plan is rejected with FST_EINVAL.
 */
fst_status fst_project_noalloc(fst_plan_t plan, const void *y, void *out, int64_t batch,
                               int64_t ld, int dtype, void *stream);
unsigned long long fst_noalloc_scratch_bytes(void);

/*
 * Launch accounting, for benchmarks (not part of the method).
 * fst_launch_count   -- number of kernels this process has launched through the
 *                       library so far (plan-time and apply kernels).
 * fst_profile_enable -- on != 0: from now on, every apply-kernel launch and the
 *                       plan-time eigen kernels (bisection, inverse iteration,
 *                       expansion) are bracketed by CUDA events on their stream;
 *                       clears earlier records.  on == 0 stops recording (and clears).
 * fst_profile_count  -- number of recorded launches.
 * fst_profile_read   -- record i: kernel name (static string), elapsed device time
 *                       in ms between its events (waits for them), and the number
 *                       of signal pairs (eigen kernels: eigenvectors) it processed.
 *                       FST_EINVAL if i is out of range.
 */
long long fst_launch_count(void);
fst_status fst_profile_enable(int on);
int fst_profile_count(void);
fst_status fst_profile_read(int i, const char **name, double *ms, long long *units);

#ifdef __cplusplus
}
#endif

#endif /* FST_GB300_H */
