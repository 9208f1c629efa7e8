/*
 * libcholdiff -- blocked Cholesky factorisation and its forward- and
 * reverse-mode derivatives on one GB300 GPU (sm_103a).
 *
 * The operations follow I. Murray, "Differentiation of the Cholesky
 * decomposition" (arXiv:1602.07527):
 *   cd_chol_fwd       Sec. 4.2 chol_blocked      (LAPACK DPOTRF):  Sigma -> L
 *   cd_chol_fwd_sens  Sec. 4.2 chol_blocked_fwd  (forward mode):   (L, Sigma_dot) -> L_dot
 *   cd_chol_rev       Sec. 4.2 chol_blocked_rev  (reverse mode):   (L, L_bar) -> tril(Sigma_bar)
 *   cd_chol_fwd_and_sens  the first two in one loop (Sec. 4.1-4.2): (Sigma, Sigma_dot) -> (L, L_dot)
 * with the problem statement of Sec. 2 (forward mode L_dot(L, Sigma_dot),
 * reverse mode Sigma_bar(L, L_bar)) and the symbolic results of Sec. 3
 * (Eqs. symfwd, symrev, symrevtril) as their exact meaning.
 *
 * ---------------------------------------------------------------------------
 * Conventions shared by every entry point
 * ---------------------------------------------------------------------------
 * Layout.  Every matrix is dense FP64, ROW-MAJOR, element (i, j) at
 *   M[i * ld + j], 0 <= i, j < n, with leading dimension ld >= n (in
 *   elements).  Pointers are DEVICE pointers on the handle's device and must
 *   be 8-byte aligned.  Only the lower triangle (i >= j) of an input is read.
 *   Only the lower triangle of an output is written, except that
 *   cd_chol_rev with CD_OUT_SYM also writes the strict upper triangle.
 *   The strictly upper triangle is otherwise neither read nor written.
 *
 * In place.  As in the paper (Sec. 4.1-4.2), each routine overwrites its
 *   input array: cd_chol_fwd turns tril(Sigma) into L, cd_chol_fwd_sens turns
 *   tril(Sigma_dot) into L_dot, cd_chol_rev turns L_bar into tril(Sigma_bar).
 *   L must not overlap the in/out array.
 *
 * Meaning of Sigma_bar.  tril(Sigma_bar) holds, for i > j, the derivative of
 *   f with respect to the tied pair Sigma_ij = Sigma_ji, and on the diagonal
 *   d f / d Sigma_ii (Eq. symrevtril).  CD_OUT_SYM instead returns the full
 *   symmetric matrix of Eq. symrev, S + S^T - diag(S), whose strict upper
 *   triangle mirrors the strict lower one.  The gradient in the convention of
 *   torch.linalg.cholesky's backward is (tril + tril^T)/2 of the CD_OUT_TRIL
 *   result.
 *
 * Triangle.  With options->uplo = CD_UPPER every "lower triangle" above reads
 *   "upper triangle" and every factor is U = L^T (Sigma = U^T U): cd_chol_fwd
 *   turns triu(Sigma) into U, cd_chol_rev turns U_bar = L_bar^T into
 *   triu(Sigma_bar) = tril(Sigma_bar)^T, cd_chol_fwd_sens turns triu(Sigma_dot)
 *   into U_dot; the strictly lower triangle is then neither read nor written
 *   (except by CD_OUT_SYM).  The library transposes the operands into
 *   workspace copies, runs the lower-triangle algorithms and transposes the
 *   results back (two extra passes over each matrix).
 *
 * Blocking.  options->nb (the paper's N_b, >= 1) is the block size; 0 picks
 *   a default.  The forward routines put a short block last and the reverse
 *   routine puts it first (top-left), as the paper does (Sec. 4.2).  Blocking
 *   only reorders rounding: every nb gives the same exact result.
 *
 * Precision.  CD_FP64 does all arithmetic in FP64.  CD_MIXED_* keeps the
 *   diagonal-tile work (factorisation, level-2 derivative loops, diagonal
 *   block inverses, the Phi / halving steps) in FP64 and runs the large
 *   off-diagonal products on BF16 tensor cores with operands split into two
 *   (x = hi + lo, 3 products) or three (6 products) BF16 terms and FP32
 *   accumulation; inputs and outputs stay FP64 in memory.
 *
 * Asynchrony and errors.  Every compute call is enqueued on `stream` (a
 *   cudaStream_t, NULL for the legacy default stream) and returns without
 *   waiting.  The return value reports argument errors (CD_EINVAL), workspace
 *   allocation failure (CD_ENOMEM) and launch failures (CD_ECUDA) detected on
 *   the host.  Errors found on the device (a bounded wait that ran out, an
 *   inconsistent tile) set the handle's device error word, readable with
 *   cd_get_last_device_error after the stream has been synchronised.
 *   n == 0 is a valid no-op.
 *
 * Ownership.  The caller owns every matrix, info array and stream.  The
 *   handle owns its workspace (grown on demand in stream order with
 *   cudaMallocAsync on the call's stream, released by cd_destroy) and must not be used by two host threads at once; calls that
 *   share a handle must be ordered on one stream (they share its workspace).
 */
#ifndef LIBCHOLDIFF_H
#define LIBCHOLDIFF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes.  Positive values are never returned by the host calls; the
 * factorisation's pivot report goes to the device `info` word instead. */
#define CD_OK 0
#define CD_EINVAL (-1)   /* bad argument: n < 0, ld < n, nb < 0, NULL pointer ... */
#define CD_ENOMEM (-2)   /* workspace allocation failed                           */
#define CD_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed          */
#define CD_ETIMEOUT (-4) /* device word: a bounded device-side wait ran out       */
#define CD_ESCRATCH (-5) /* cd_chol_rev_noalloc: problem larger than its fixed scratch */

typedef enum {
  CD_FP64 = 0,          /* all FP64 (DFMA)                                    */
  CD_MIXED_BF16X3 = 1,  /* products as hi*hi + hi*lo + lo*hi, BF16 in, FP32 acc */
  CD_MIXED_BF16X6 = 2,  /* three-term split, 6 BF16 products, FP32 accumulate  */
  CD_MIXED_FIXED4 = 3   /* factorisation products on fixed-point slices: four
                           BF16 slices per element sharing one exponent per
                           row, 13 products, leading sums exact in FP32 over
                           windows of 512 of K and carried exactly in 64-bit
                           integers (operands rounded to 2^-32 of their row maxima);
                           derivative passes as CD_MIXED_BF16X6              */
} cd_precision;

typedef enum {
  CD_OUT_TRIL = 0, /* tril(Sigma_bar), Eq. symrevtril; strict upper untouched */
  CD_OUT_SYM = 1   /* full symmetric Sigma_bar of Eq. symrev                   */
} cd_output;

typedef enum {
  CD_DIAG_AUTO = 0,     /* the faster on GB300: currently CD_DIAG_SYMBOLIC       */
  CD_DIAG_LEVEL2 = 1,   /* one-CTA level-2 loop on the tile (Sec. 4.1)           */
  CD_DIAG_SYMBOLIC = 2  /* Eq. symrevtril / Eq. symfwd as FP64 products with the
                           diagonal block's inverse, spread over many CTAs     */
} cd_diag;

typedef enum {
  CD_LOWER = 0, /* Sigma = L L^T, lower triangles referenced (the paper's form) */
  CD_UPPER = 1  /* Sigma = U^T U with U = L^T, upper triangles referenced
                   (LAPACK's uplo = 'U'); see "Triangle" above             */
} cd_uplo;

typedef struct {
  int nb;               /* block size N_b; 0 = library default                 */
  int prec;             /* a cd_precision value                                */
  int out;              /* a cd_output value (cd_chol_rev only)                */
  int diag;             /* a cd_diag value: the diagonal-block routine of the
                           reverse and forward-sensitivity passes (Sec. 4.2
                           allows either; both give the exact result)        */
  int uplo;             /* a cd_uplo value                                     */
  long long spin_limit; /* bound on device-side wait iterations; 0 = default   */
} cd_options;

typedef struct cd_handle cd_handle;

/* Create a handle bound to CUDA device `device`.  *h receives the handle.
 * Returns CD_OK, CD_EINVAL (h NULL or bad device) or CD_ECUDA. */
int cd_create(cd_handle **h, int device);

/* Release the handle and its workspace.  The caller must first make sure no
 * work enqueued with the handle is still running.  NULL is accepted. */
int cd_destroy(cd_handle *h);

/* Fill *opt with the defaults (nb 0, CD_FP64, CD_OUT_TRIL, default spin limit). */
void cd_options_default(cd_options *opt);

/* Bytes of workspace a call of size n_max with these options may use; a
 * caller may pre-grow the handle with cd_reserve to keep later calls from
 * allocating. */
int cd_workspace_size(const cd_handle *h, int n_max, const cd_options *opt, size_t *bytes);

/* Bytes of workspace any batched call over the `batch` problem sizes n[]
 * (host array) with these options may use: the bound the handle's workspace
 * grows to for that batch.  A caller that keeps a handle's workspace at a
 * fixed size (cd_reserve) and admits only batches whose bound fits keeps the
 * library from allocating during its calls. */
int cd_workspace_size_batched(const cd_handle *h, int batch, const int *n, const cd_options *opt, size_t *bytes);

/* Grow the handle's workspace to `bytes` now if it holds less (exactly that
 * many bytes; returns when it is allocated).  Growth inside the compute calls
 * adds an eighth as headroom. */
int cd_reserve(cd_handle *h, size_t bytes);

/* Bytes of workspace the handle holds now. */
int cd_workspace_bytes(const cd_handle *h, size_t *bytes);

/*
 * Blocked Cholesky factorisation (Sec. 4.2 chol_blocked, mirroring DPOTRF):
 * overwrites tril(A) (holding tril(Sigma), n x n, leading dimension lda)
 * with L, Sigma = L L^T.  info (device int*, may be NULL) receives 0 on
 * success or the 1-based index j of the first column whose pivot
 * Sigma_jj - sum_k L_jk^2 is not positive or not a number (LAPACK's info);
 * L is then unspecified from that column on.  No pivoting.
 */
int cd_chol_fwd(cd_handle *h, int n, double *A, long long lda,
                const cd_options *opt, void *stream, int *info);

/*
 * Reverse mode (Sec. 4.2 chol_blocked_rev; exact meaning Eq. symrevtril):
 * given the factor L (lower, n x n, ldl) and tril(Abar) = L_bar (n x n,
 * lda), overwrites tril(Abar) with tril(Sigma_bar) (or the full symmetric
 * Sigma_bar of Eq. symrev with CD_OUT_SYM).  L's diagonal must be nonzero.
 */
int cd_chol_rev(cd_handle *h, int n, const double *L, long long ldl,
                double *Abar, long long lda, const cd_options *opt, void *stream);

/*
 * Forward mode (Sec. 4.2 chol_blocked_fwd; exact meaning Eq. symfwd):
 * given L and tril(Adot) = tril(Sigma_dot) of the symmetric perturbation
 * Sigma_dot, overwrites tril(Adot) with L_dot = L Phi(L^{-1} Sigma_dot L^{-T}).
 */
int cd_chol_fwd_sens(cd_handle *h, int n, const double *L, long long ldl,
                     double *Adot, long long lda, const cd_options *opt, void *stream);

/*
 * Factorisation and forward mode in one pass (Sec. 4.1 and Sec. 4.2: the
 * forward-mode updates may be accumulated in the same loop as the
 * factorisation).  On entry tril(A) = tril(Sigma) (n x n, lda) and
 * tril(Adot) = tril(Sigma_dot) (n x n, ldadot); on exit tril(A) = L as
 * cd_chol_fwd and tril(Adot) = L_dot as cd_chol_fwd_sens would give from that
 * L, Eq. symfwd.  A and Adot must not overlap.  info as for cd_chol_fwd; on a
 * non-positive pivot both outputs are unspecified from that column on.
 * Blocking, precision (split-BF16 products for CD_MIXED_*) and the diagonal
 * routine follow options as for the two separate calls.  Both halves use the
 * factorisation's block size; each forward-mode block step is issued as soon
 * as the factorisation has finished its block column and runs beside it on a
 * second pair of the handle's internal streams, so the call takes less time
 * than the two separate calls.
 */
int cd_chol_fwd_and_sens(cd_handle *h, int n, double *A, long long lda, double *Adot, long long ldadot,
                         const cd_options *opt, void *stream, int *info);

/*
 * Batched variants over `batch` independent problems of ragged sizes.
 * n, A/L/Abar/Adot pointers and leading dimensions are HOST arrays of length
 * `batch` (the pointers inside are device pointers); problem b has size
 * n[b] >= 0 and leading dimension ld[b] >= n[b].  Problems are independent
 * (Sec. 2: each is its own x -> Sigma -> L -> f chain); their work is
 * interleaved on the device so small problems share the GPU.  info (device
 * int array of length batch, may be NULL) receives each factorisation's info.
 * Results equal those of the single-problem calls with the same options.
 */
int cd_chol_fwd_batched(cd_handle *h, int batch, const int *n, double *const *A,
                        const long long *lda, const cd_options *opt, void *stream, int *info);
int cd_chol_rev_batched(cd_handle *h, int batch, const int *n, const double *const *L,
                        const long long *ldl, double *const *Abar, const long long *lda,
                        const cd_options *opt, void *stream);
int cd_chol_fwd_sens_batched(cd_handle *h, int batch, const int *n, const double *const *L,
                             const long long *ldl, double *const *Adot, const long long *lda,
                             const cd_options *opt, void *stream);
int cd_chol_fwd_and_sens_batched(cd_handle *h, int batch, const int *n, double *const *A,
                                 const long long *lda, double *const *Adot, const long long *ldadot,
                                 const cd_options *opt, void *stream, int *info);

/*
 * Explicit Jacobian of the factor (Eq. delements), for analysis and testing:
 *   J[((i n + j) n + k) n + l] = d L_ij / d Sigma_kl   for i >= j, k >= l,
 * where Sigma_kl and Sigma_lk (k != l) are one tied input, as in Eq. symrev;
 * every other entry is 0.  L (n x n, ldl, lower triangle read) is the factor;
 * J is a caller-owned device array of n^4 doubles.  Theta(n^4) time and
 * memory (n = 128 needs 2.1 GB): this is not the blocked hot path, whose
 * Jacobian-vector products are cd_chol_fwd_sens and cd_chol_rev.  The
 * handle's workspace holds L^{-1} and the n^3 partial sums of the formula.
 * FP64 only.  Asynchronous on stream.
 */
int cd_chol_jacobian(cd_handle *h, int n, const double *L, long long ldl, double *J, void *stream);

/*
 * Reverse mode without any allocation (no counterpart in the paper: this is a
 * service for callers, not a step of the method).
 *
 * Some callers cannot allocate device memory when they need the gradient:
 * code running inside a region whose allocations are forbidden (a custom
 * allocator's callbacks, a framework that owns all device memory), or an
 * embedding that must never let the library grow its footprint.  They cannot
 * use cd_chol_rev, whose handle allocates its workspace on demand, nor even
 * cd_create.  This entry point computes the same result as cd_chol_rev with
 * CD_FP64 for one problem, with no handle: all of its scratch (inverses of
 * L's diagonal blocks, the solved panel, split-K partial sums) lives in one
 * fixed 8 MiB device array inside the library, which every GPU that loads the
 * library holds until the process exits.  The call performs no cudaMalloc,
 * cudaFree or other allocating call.
 *
 *   n       problem size, 0 <= n <= CD_NOALLOC_MAX_N (2048); larger n returns
 *           CD_ESCRATCH and does nothing.
 *   L, ldl  device factor as for cd_chol_rev; Abar, lda in/out as for cd_chol_rev.
 *   nb      block size, 0 (default) or 1..CD_NOALLOC_MAX_NB (128).
 *   out     CD_OUT_TRIL or CD_OUT_SYM.
 *   stream  cudaStream_t of the call; runs on the current CUDA device.
 *
 * The first call on a device looks up the array's device address and
 * prepares the kernels (no allocation); make that first call before any
 * stream capture.  Every call on a device shares the one array and each call
 * leaves its contents behind; no word of it needs to start at zero, since a
 * call writes every scratch word before reading it.  Calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on
 * the array and give wrong results: order them.  Results agree with
 * cd_chol_rev to rounding (the split-K partition may differ).
 */
#define CD_NOALLOC_MAX_N 2048
#define CD_NOALLOC_MAX_NB 128
int cd_chol_rev_noalloc(int n, const double *L, long long ldl, double *Abar, long long lda,
                        int nb, int out, void *stream);

/*
 * Diagnostic: the tensor-core products used by the CD_MIXED_* paths, exposed
 * so that they can be tested alone (no counterpart in the paper).  C (M x N,
 * ldc) = A B^T with A (M x K, lda) and B (N x K, ldb), all FP64 row-major
 * device matrices; prec is CD_MIXED_BF16X3 or CD_MIXED_BF16X6 (split-BF16
 * product) or CD_MIXED_FIXED4 (fixed-point slice product, each row's exponent
 * taken from its maximum); lower != 0 (requires M == N) writes only i >= j.
 * Uses the handle's workspace; asynchronous on stream.
 */
int cd_mixed_gemm_debug(cd_handle *h, int M, int N, int K, const double *A, long long lda, const double *B,
                        long long ldb, double *C, long long ldc, int prec, int lower, void *stream);

/*
 * Diagnostic (no counterpart in the paper): the FP64 reciprocal and square
 * root that the diagonal factorisation uses on its pivots, applied to the n
 * device values x[i] > 0: recip[i] ~ 1 / x[i] (an FP32 seed refined by one
 * Householder step of order 2), sq[i] ~ sqrt(x[i]) and rsq[i] ~ 1 / sqrt(x[i])
 * (Goldschmidt's iteration from an FP32 seed).  Zero, subnormal, infinite
 * and NaN inputs take the platform's division and square root.  Device
 * arrays of n doubles; asynchronous on stream.
 */
int cd_debug_fp64_helpers(cd_handle *h, int n, const double *x, double *recip, double *sq, double *rsq,
                          void *stream);

/*
 * Measurement support (no counterpart in the paper): the rate of the FP64
 * pipe.  Launches 4 CTAs of 256 threads per SM, each thread running `iters`
 * rounds of register-only FP64 work: kind 0 a 4 x 2 outer product of FMAs
 * (DFMA, the instruction of the FP64 products here), kind 1 four chains of
 * the FP64 matrix instruction mma.sync m8n8k4 (DMMA).  *flops receives the
 * floating-point operations launched (2 per multiply-add); the caller times
 * the launch on `stream`.  Returns CD_EINVAL for a bad kind or iters < 1.
 */
int cd_debug_fp64_probe(cd_handle *h, int kind, long long iters, void *stream, double *flops);

/*
 * Scheduling knob (no counterpart in the paper).  Every call runs its
 * diagonal chain on one internal stream and the step's independent bulk
 * product on another, both forked from and joined back into the caller's
 * stream; the one-loop pass runs its sensitivity steps on a
 * second such pair.  This sets their CUDA stream priorities (clamped to the
 * device's range; lower numbers are higher priority; defaults: greatest for
 * the chains, least for the bulk).  Handles serving latency-critical work can
 * be raised above others that share the GPU.  Synchronises the handle's
 * device.
 */
int cd_set_priorities(cd_handle *h, int chain_priority, int bulk_priority);

/*
 * Test hook for the device-side failure path (no counterpart in the paper).
 * Runs one small tensor-core product whose first load barrier expects 16
 * bytes more than its copy delivers: the copy completes, nothing else is in
 * flight, and the consumer's bounded wait gives up after about 2 s.  The
 * kernel then sets the handle's device error word to CD_ETIMEOUT, frees its
 * tensor memory and exits without writing its output; the context stays
 * usable.  Read the word with cd_get_last_device_error.
 */
int cd_debug_wait_timeout(cd_handle *h, void *stream);

/* Read and clear the handle's device error word (synchronises the handle's
 * device).  *code receives CD_OK or a negative CD_* code. */
int cd_get_last_device_error(cd_handle *h, int *code);

/* Number of kernel launches this handle has issued since creation (a
 * counter kept on the host; used to report launch counts). */
long long cd_launch_count(const cd_handle *h);

/* Library version string. */
const char *cd_version(void);

/*
 * Kernel profiler (measurement support; the paper has no counterpart).
 * While enabled, the handle records a CUDA event pair around every kernel it
 * launches, tagged with the kernel kind and that launch's algorithmic work
 * (useful flops of the products it computes and the minimum bytes it must
 * move).  cd_profile_read synchronises the handle's device, aggregates the
 * recorded launches per kind into out[0..*count) (at most `max` kinds, in
 * order of total time, largest first) and clears the record.  Recording
 * costs one event pair per launch; it does not change any result.
 */
typedef struct {
  char name[48];      /* kernel kind, e.g. "gemm_f64<SYM2,N>"          */
  long long launches; /* launches recorded                              */
  double ms;          /* sum of per-launch device time (CUDA events)    */
  double flops;       /* sum of algorithmic flops                       */
  double bytes;       /* sum of algorithmic bytes                       */
} cd_kernel_stat;

int cd_profile_enable(cd_handle *h, int on);
int cd_profile_read(cd_handle *h, cd_kernel_stat *out, int max, int *count);

/*
 * The recorded launches one by one, in launch order, without clearing them
 * (call it before cd_profile_read): out[0..*count) (at most `max`) gets each
 * launch's kind, the stream it ran on (0 = the caller's stream, 1 = the
 * handle's side stream) and its start and end in milliseconds from the
 * first recorded launch's start.  Synchronises the handle's device.  Shows
 * how the side stream's products overlap the diagonal chain.
 */
typedef struct {
  char name[48];
  int stream;
  double start_ms, end_ms;
} cd_launch_rec;

int cd_profile_timeline(cd_handle *h, cd_launch_rec *out, int max, int *count);

#ifdef __cplusplus
}
#endif

#endif /* LIBCHOLDIFF_H */
