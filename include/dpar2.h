/*
 * dpar2.h -- C ABI of the GB300 DPar2 library (libdpar2.so).
 *
 * DPar2 (Jang & Kang, "DPar2: Fast and Scalable PARAFAC2 Decomposition for
 * Irregular Dense Tensors", arXiv 2203.12798) fits the PARAFAC2 model
 * X_k ~ Q_k H S_k V^T (Def. 1, Sec. II-C; objective Eq. PARAFAC2_reform) to
 * an irregular tensor {X_k}, k = 1..K, X_k of size I_k x J, by
 *   1. compressing every slice with a randomized SVD, X_k ~ A_k B_k C_k^T
 *      (Alg. 1; Eq. fstage_svd; Alg. 3 first loop),
 *   2. compressing M = [C_1 B_1 ... C_K B_K] (J x KR) with a second
 *      randomized SVD, M ~ D E F^T (Eq. matricization_svd),
 *   3. running ALS on the compressed slices A_k F^(k) E D^T (Eq. Xk_final;
 *      Sec. III-C..E; Alg. 3 repeat loop): a batched R x R SVD per slice
 *      (Eq. q_k), the MTTKRPs of Lemmas 1-3 and the H / V / W updates.
 *
 * Conventions for every entry point
 *   - All matrices are row-major.  "device" pointers are CUDA global memory
 *     on the context's device; "host" pointers are ordinary host memory.
 *   - Every call enqueues its work on `stream` (a cudaStream_t, NULL = the
 *     legacy default stream) and returns after that work has completed; the
 *     caller's buffers may be reused when the call returns.
 *   - Every call returns a dpar2_status; nothing throws across the ABI.  On
 *     failure dpar2_last_error(ctx) gives a one-line explanation.  Argument
 *     and shape checks happen on the host before any launch.  Faults found
 *     on the device (non-finite values, a bounded wait that ran out) are
 *     recorded in a device status word and reported by the call.
 *   - The library owns dpar2_ctx and dpar2_comp objects (free them with
 *     dpar2_destroy / dpar2_comp_free); everything else is caller-owned.
 *   - Precision: X may be FP32, BF16 or FP16 (storage and multiplication
 *     type, FP32 accumulation).  The Gram matrices of both CholeskyQR2 steps
 *     are double-float sums of exact FP32 products (about 48 significant
 *     bits), stored in FP64; the first step's Cholesky is FP64, the second's
 *     (a matrix within ~1e-6 of the identity) FP32.  The R x R Gram-Hadamard
 *     normal equations of the H, V and W updates are inverted and applied in
 *     FP64.  Norm and fitness reductions are FP64.  All factor outputs are
 *     FP32.
 */
#ifndef DPAR2_H_
#define DPAR2_H_

#include <stddef.h>
#include <stdint.h>

#if defined(DPAR2_BUILD) && defined(__GNUC__)
#define DPAR2_API __attribute__((visibility("default")))
#else
#define DPAR2_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DPAR2_OK = 0,
  DPAR2_ERR_INVALID_ARG = 1, /* null pointer, bad option value, misaligned buffer */
  DPAR2_ERR_SHAPE = 2,       /* K, J, R, offsets or ld inconsistent */
  DPAR2_ERR_CUDA = 3,        /* a CUDA runtime / driver call failed */
  DPAR2_ERR_NUMERICAL = 4,   /* non-finite values met on the device */
  DPAR2_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  DPAR2_ERR_OOM = 6,         /* device memory allocation failed */
  DPAR2_ERR_UNSUPPORTED = 7  /* option combination not implemented */
} dpar2_status;

typedef enum { DPAR2_F32 = 0, DPAR2_BF16 = 1, DPAR2_F16 = 2 } dpar2_dtype;

/* dpar2_options.flags */
#define DPAR2_FLAG_PER_SLICE 0x1u /* stage 1 launched once per slice (the plain form) */
#define DPAR2_FLAG_NO_GRAPH 0x2u  /* do not capture the ALS loop in a CUDA graph */
#define DPAR2_FLAG_GENERIC 0x4u   /* CUDA-core stage-1 kernels even for 16-bit X */
#define DPAR2_FLAG_DROP_M 0x8u    /* free M after stage 2 (identity fitness then needs X) */
#define DPAR2_FLAG_COLD_QSTEP 0x10u /* Q-step Jacobi from the identity every iteration (no warm start) */
#define DPAR2_FLAG_FIVE_LAUNCH 0x20u /* ALS iterations as five launches with single-block H and V updates
                                        (the form used for R > 32) instead of three */
#define DPAR2_FLAG_NO_PERSIST 0x40u  /* ALS iterations as launches per iteration instead of the one
                                        persistent launch used when tol < 0, R <= 20 and the slices fit
                                        one pass of its warps (K <= (SMs - 1) x 54 at R <= 10,
                                        (SMs - 1) x 8 at R <= 20) */

typedef struct {
  int R;          /* target rank (Alg. 1 / Alg. 3 parameter), 1 <= R <= 64 */
  int p;          /* oversampling s of Alg. 1: sketch width l = R + p <= 64 */
  int q;          /* power-iteration exponent q of Alg. 1 (stage 1 and stage 2) */
  uint64_t seed;  /* Philox seed of the Gaussian test matrices and of V_0 */
  int max_iter;   /* maximum ALS iterations (Alg. 3 repeat loop) */
  double tol;     /* stop when e_prev - e <= tol * e_prev; tol < 0: run max_iter */
  int schedule;   /* slice-to-CTA schedule of the tensor-core projection: 0 = work items
                     round-robin over the CTAs, 1 = longest slices first, each item onto
                     the least-loaded CTA; -1 = autotuned (both timed on the first
                     compression of a problem shape, the faster kept by the context) */
  unsigned flags; /* DPAR2_FLAG_* */
  int proj_cols;  /* X columns per work item of the tensor-core projection: 0 = the widest
                     that TMEM holds double-buffered (512 for l <= 21, 256 for l <= 32, 128
                     above), or for l <= 21 also 256; with schedule = -1 and proj_cols = 0
                     both widths are timed with both schedules on the first compression of a
                     problem shape and the fastest pair is kept.  Every width computes each
                     column of B_k identically and ||X_k||^2 from the same FP32 partial sums
                     (their FP64 total differs at the FP64 rounding level) */
} dpar2_options;

typedef struct dpar2_ctx dpar2_ctx;
typedef struct dpar2_comp dpar2_comp;

/* Device views of a compressed representation (library-owned memory, valid
 * until dpar2_comp_free).  Shapes:
 *   A       sum(I_k) x R   stage-1 left factors A_k stacked by slice (Eq. fstage_svd)
 *   Bk      K x R          stage-1 singular values (diagonal of B_k)
 *   Ms      3 x KR x Jq    M^T in three BF16 parts whose sum is M exactly (part p
 *                          at Ms + p KR Jq elements; row k R + r holds column r of
 *                          M_k = C_k B_k, the k-th J x R block of M; Jq = J rounded
 *                          up to 64, columns past J zero), or NULL; dpar2_comp_m
 *                          reassembles M in FP32
 *   D       J x R          stage-2 left factor (Eq. matricization_svd)
 *   E       R              stage-2 singular values
 *   Ft      K x R x R      F^(k) E, the k-th R x R block of F times E (Eq. verticalF)
 *   xnorm2  K              ||X_k||_F^2 (FP64)
 *   offsets K + 1          slice row offsets (int64, device copy)            */
typedef struct {
  int K, J, R, ell;
  int Jq;    /* J rounded up to 64 */
  int64_t N; /* sum_k I_k */
  const int64_t* offsets;
  const float* A;
  const float* Bk;
  const void* Ms;
  const float* D;
  const float* E;
  const float* Ft;
  const double* xnorm2;
  int32_t* rank1; /* per-slice numerical rank of the stage-1 sketch (device, K) */
} dpar2_comp_view;

/* Fill *opt with R=10, p=10, q=0, seed=0, max_iter=32, tol=-1, schedule=-1, proj_cols=0. */
DPAR2_API dpar2_status dpar2_options_default(dpar2_options* opt);

/* Create a context bound to CUDA device `device`.  Owns scratch memory that
 * grows on demand and is reused across calls. */
DPAR2_API dpar2_status dpar2_create(dpar2_ctx** ctx, int device);
DPAR2_API void dpar2_destroy(dpar2_ctx* ctx);
DPAR2_API const char* dpar2_last_error(const dpar2_ctx* ctx);
/* Information bits of the last call's device status word (not errors; the
 * paper has no counterpart): a CholeskyQR step dropped a numerically
 * dependent sketch column, a Jacobi solver stopped at its sweep cap, a
 * Gram-Hadamard solve fell back to the eigen pseudoinverse.  0 for a null ctx. */
#define DPAR2_INFO_RANK_DROP 4
#define DPAR2_INFO_SWEEP_CAP 8
#define DPAR2_INFO_PINV 16
DPAR2_API int dpar2_last_info(const dpar2_ctx* ctx);
/* Number of kernels this library has launched since it was loaded, over all
 * contexts and threads (kernels run from a CUDA graph count once per graph
 * launch).  The paper has no counterpart; for accounting, e.g. launches per
 * fit: read it before and after the calls of interest, with no other thread
 * using the library meanwhile. */
DPAR2_API long long dpar2_kernel_launches(void);

/* Fill out[0..n) (device, float32) with the Gaussian stream (seed, stream_id):
 * Philox4x32-10 (Salmon et al. SC'11) with counter (n/4 lo, n/4 hi, stream_id, 0)
 * and key (seed lo, seed hi), Box-Muller on word pairs.  round16 != 0 rounds
 * every value to the nearest bf16 and flushes |x| < 2^-14 to zero so that it
 * is exact in fp32, bf16 and fp16. */
DPAR2_API dpar2_status dpar2_gaussian(dpar2_ctx* ctx, uint64_t seed, uint32_t stream_id, int64_t n, float* out,
                            int round16, void* stream);
/* The raw 32-bit words 0..n-1 of the same Philox stream (device, uint32). */
DPAR2_API dpar2_status dpar2_philox_words(dpar2_ctx* ctx, uint64_t seed, uint32_t stream_id, int64_t n, uint32_t* out,
                                void* stream);

/* Two-stage compression (Sec. III-B; Alg. 3 lines "compress slices", "M <-",
 * "SVD(M)").
 *   K, J         number of slices and columns (K >= 1, J >= 1)
 *   row_offsets  host, K+1 int64, offsets[0] = 0, I_k = offsets[k+1]-offsets[k] >= 1
 *   X            device, sum(I_k) rows of ldx elements of `dtype`; X_k is rows
 *                offsets[k] .. offsets[k+1]-1, columns 0..J-1.  ldx >= J and
 *                ldx * sizeof(dtype) must be a multiple of 16 bytes, X 16-byte
 *                aligned (a multiple of 32 bytes is faster: every 512-column
 *                block of a row then starts on a DRAM sector boundary).  Read
 *                only; must stay valid until the call returns.
 *   opt          R, p, q, seed, schedule, flags are used.  Requires R <= J,
 *                R + p <= min(J, 64).
 *   omega        device J x (R+p) float32 test matrix of stage 1, or NULL for
 *                the Gaussian stream (opt->seed, 0) rounded as in dpar2_gaussian.
 *                For 16-bit X its values are used rounded to that type.
 *   omega2       device (K R) x (R+p) float32 test matrix of stage 2, or NULL
 *                for the Gaussian stream (opt->seed, 1).
 *   out          receives a new library-owned compressed representation.
 * Slices with I_k < R + p (or rank-deficient slices) keep only their
 * numerical rank; the remaining columns of A_k, entries of B_k and columns
 * of C_k B_k are zero. */
DPAR2_API dpar2_status dpar2_compress(dpar2_ctx* ctx, int K, int J, const int64_t* row_offsets, const void* X,
                            int64_t ldx, dpar2_dtype dtype, const dpar2_options* opt, const float* omega,
                            const float* omega2, dpar2_comp** out, void* stream);

/* The same two-stage compression for a tensor held in host memory (Sec. III-B;
 * every slice is compressed from its own rows by Alg. 1, so stage 1 can run
 * chunk by chunk).  The slices are cut into chunks of whole slices of about
 * chunk_bytes of X; each chunk is copied to the device once, on a copy stream
 * of the context, while the previous chunk's stage 1 runs, so X crosses the
 * host link once and the copies hide the stage-1 work.  X need not fit in
 * device memory unless X_dev is given.
 *   X_host       host, sum(I_k) rows of J elements of `dtype`, packed (row
 *                stride J).  Pinned (page-locked) memory gives asynchronous,
 *                full-rate copies; pageable memory works but copies slowly.
 *                Read only; must stay valid until the call returns.
 *   X_dev        device buffer of sum(I_k) rows of ldx elements that receives X
 *                (columns J..ldx-1 zero), for later calls that read X again
 *                (dpar2_reconstruct_error's streamed mode); or NULL: chunk
 *                buffers of the context are used and X is not kept.  ldx: as for
 *                dpar2_compress (ignored when X_dev is NULL).
 *   chunk_bytes  target bytes of X per chunk (0: 2 GB); a chunk holds at
 *                least one slice.  Context scratch: three staging buffers of
 *                the largest chunk (unless ldx == J) and, without X_dev, three
 *                chunk buffers of it; copies run up to three chunks ahead.
 * Other arguments, outputs and errors as dpar2_compress.  The result is the
 * compression dpar2_compress computes from the same X (the same kernels per
 * slice; chunks of fewer than 256 slices sum the CholeskyQR Grams of their
 * slices in a different order, a difference at rounding level).  Only the
 * DPAR2_PH_COMPRESS phase time is recorded. */
DPAR2_API dpar2_status dpar2_compress_host(dpar2_ctx* ctx, int K, int J, const int64_t* row_offsets,
                                           const void* X_host, dpar2_dtype dtype, const dpar2_options* opt,
                                           const float* omega, const float* omega2, void* X_dev, int64_t ldx,
                                           size_t chunk_bytes, dpar2_comp** out, void* stream);

/* ALS iterations on the compressed slices (Alg. 3 repeat loop, Sec. III-C..E).
 *   comp          from dpar2_compress
 *   opt           R must equal the compression's R; max_iter, tol, seed, flags used
 *   V0            device J x R initial V, or NULL for the Gaussian stream (seed, 3);
 *                 H_0 = I_R and S_k = I (W_0 = ones) always
 *   H, V, W       device outputs R x R, J x R, K x R (S_k = diag(W(k,:)))
 *   Upol          device output K x R x R, Z_k P_k^T of the last Q-step (Eq. q_k), or NULL
 *   U             device output sum(I_k) x R, U_k = A_k Z_k P_k^T H (Alg. 3 last loop), or NULL
 *   loss_history  host output of max_iter doubles (e after each iteration), or NULL
 *   iters_run     host output, iterations performed, or NULL
 *   fitness       host output: 1 - sum||X_k - X^_k||^2 / sum||X_k||^2 (Sec. IV-A)
 *                 through the exact stage-1 identity (needs M), or NULL */
DPAR2_API dpar2_status dpar2_fit(dpar2_ctx* ctx, const dpar2_comp* comp, const dpar2_options* opt, const float* V0,
                       float* H, float* V, float* W, float* Upol, float* U, double* loss_history,
                       int* iters_run, double* fitness, void* stream);

/* Squared reconstruction error and fitness (Sec. IV-A) of the model
 * X^_k = A_k Upol_k H S_k V^T.
 *   X == NULL  identity mode: ||X_k||^2 - 2 <B_k C_k^T, Upol_k H S_k V^T> + ||Upol_k H S_k V^T||^2,
 *              exact because A_k^T X_k = B_k C_k^T for the randomized SVD (needs M).
 *   X != NULL  streamed mode: reads X again (same layout rules as dpar2_compress)
 *              and sums ||X_k - A_k (Upol_k H S_k V^T)||^2 row by row.
 *   H, V, W    device R x R, J x R, K x R;  Upol device K x R x R, or NULL to
 *              recompute it with one Q-step from H, V, W.
 *   sq_err, fitness  host outputs (either may be NULL). */
DPAR2_API dpar2_status dpar2_reconstruct_error(dpar2_ctx* ctx, const dpar2_comp* comp, const void* X, int64_t ldx,
                                     dpar2_dtype dtype, const float* H, const float* V, const float* W,
                                     const float* Upol, double* sq_err, double* fitness, void* stream);

/* Identity-mode dpar2_reconstruct_error (X == NULL, Upol given) that
 * allocates no device memory.  The paper has no counterpart: this variant
 * exists for callers that must not allocate during a call.  Its scratch is a
 * fixed array of DPAR2_NOALLOC_SCRATCH_BYTES (18 MiB) in the library's device
 * image, one per device, enough for K R^2 <= 4,194,304 (for example K = 8000
 * slices at R <= 22); larger problems are rejected with DPAR2_ERR_INVALID_ARG
 * before anything is launched.  Every call looks up the array's address on
 * the context's device (cudaGetSymbolAddress, which allocates nothing), so a
 * device context that was reset between calls is handled; the first call on
 * a device may also load the library's device code there, so make that first
 * call before any stream capture.  No scratch word has to start at zero: every word a call
 * reads is written earlier in the same call.  All calls on a device share the
 * one array, so calls that overlap in time (other host threads, other
 * contexts on the same device) race on it and must be serialised by the
 * caller; consecutive calls are safe since each call has finished its device
 * work when it returns.
 *   H, V, W, Upol    device R x R, J x R, K x R, K x R x R (as dpar2_reconstruct_error)
 *   sq_err, fitness  host outputs (either may be NULL) */
#define DPAR2_NOALLOC_SCRATCH_BYTES (18u << 20)
#define DPAR2_NOALLOC_MAX_KRR (1u << 22) /* largest K R^2 accepted */
DPAR2_API dpar2_status dpar2_reconstruct_error_noalloc(dpar2_ctx* ctx, const dpar2_comp* comp, const float* H,
                                                       const float* V, const float* W, const float* Upol,
                                                       double* sq_err, double* fitness, void* stream);

/* Copy `rows` rows of J elements of `dtype` from host memory (rows packed,
 * row stride J; pinned memory gives asynchronous, full-bandwidth copies) into
 * the device layout dpar2_compress reads (row stride ldx elements, X_dev
 * 16-byte aligned).  Columns J..ldx-1 of X_dev are set to zero.  ldx == J: one
 * copy; otherwise contiguous chunks through four device staging buffers (4 x ~128 MB
 * of context scratch) on two copy streams, each re-pitched on the device while the
 * next ones copy. */
DPAR2_API dpar2_status dpar2_upload_rows(dpar2_ctx* ctx, const void* X_host, int64_t rows, int J, dpar2_dtype dtype,
                                         void* X_dev, int64_t ldx, void* stream);

/* Inspection of the context's scratch buffers after a call (for tests and
 * debugging): *ptr / *bytes receive the device address and size of the
 * buffer `name` ("Y": sketch rows, N x LP float32, holding Q1 = Y R1^+ after
 * CholeskyQR2; "M2": K x LP x LP float32; "B1": K x LP x Jp float32 projections
 * Q1^T X_k; "GB": K x LP x LP float64 Grams B1 B1^T; "T": K x LP x R float32;
 * LP = round_up(R + p, 8), Jp = round_up(J, 4)).  Contents are valid until
 * the next call on the context; DPAR2_ERR_INVALID_ARG for an unknown name. */
DPAR2_API dpar2_status dpar2_scratch(dpar2_ctx* ctx, const char* name, void** ptr, size_t* bytes);

/* Phase timing.  With timing enabled the library records CUDA events on its
 * work stream around the phases of every dpar2_compress / dpar2_fit call;
 * dpar2_last_timings copies the durations (milliseconds) of the phases of
 * the most recent calls into ms[0..n) and returns how many it wrote.  Phase
 * indices: */
#define DPAR2_PH_SKETCH 0   /* stage-1 sketch pass Y = X Omega over all slices */
#define DPAR2_PH_QR 1       /* CholeskyQR2 of the sketches (+ power iterations) */
#define DPAR2_PH_PROJECT 2  /* stage-1 projection pass B = Q^T X and ||X_k||^2 */
#define DPAR2_PH_SMALL 3    /* small SVDs, blocks C_k B_k of M, A_k */
#define DPAR2_PH_STAGE2 4   /* randomized SVD of M -> D, E, F */
#define DPAR2_PH_COMPRESS 5 /* whole dpar2_compress */
#define DPAR2_PH_ALS 6      /* the ALS iterations of dpar2_fit */
#define DPAR2_PH_OUTPUT 7   /* V, U, fitness of dpar2_fit */
#define DPAR2_NUM_PHASES 8
DPAR2_API dpar2_status dpar2_set_timing(dpar2_ctx* ctx, int enable);
DPAR2_API int dpar2_last_timings(const dpar2_ctx* ctx, double* ms, int n);

/* Bytes of the preprocessed data in the sense of Theorem 2 (A_k, F^(k), D,
 * E stored as float32): 4 (sum_k I_k R + K R^2 + J R + R). */
DPAR2_API size_t dpar2_comp_bytes(const dpar2_comp* comp);
/* Device bytes the object actually holds (adds B_k, M, ||X_k||^2, offsets). */
DPAR2_API size_t dpar2_comp_device_bytes(const dpar2_comp* comp);
DPAR2_API dpar2_status dpar2_comp_view_get(const dpar2_comp* comp, dpar2_comp_view* view);
/* The tensor-core projection's slice-to-CTA schedule (0 round-robin, 1
 * longest slices first) and X columns per work item used by the context's
 * last compression (the autotuned pair when it was tuned); -1 / 0 if none ran
 * (FP32 X, CUDA-core passes).  Host values; the paper has no counterpart. */
DPAR2_API dpar2_status dpar2_projection_config(const dpar2_ctx* ctx, int* schedule, int* cols);
/* M (device K x J x R FP32, block k = C_k B_k) reassembled from the three BF16
 * parts of M^T the compression holds (inspection; ordered after the work
 * already queued on `stream`, NULL = the default stream, and complete when the
 * call returns).  Errors: INVALID_ARG for a null argument or a compression
 * whose M was dropped (DPAR2_FLAG_DROP_M). */
DPAR2_API dpar2_status dpar2_comp_m(dpar2_ctx* ctx, const dpar2_comp* comp, float* M, void* stream);
DPAR2_API void dpar2_comp_free(dpar2_comp* comp);

/* Learned sketch (range-finder loss of a trainable test matrix Omega).
 *
 * Alg. 1 replaces slice X_k by Q_k Q_k^T X_k, Q_k an orthonormal basis of the
 * sketch Y_k = X_k Omega; the loss of Omega is what it leaves out:
 *   L(Omega) = (1/K) sum_k ||X_k - Y_k Y_k^+ X_k||_F^2 / ||X_k||_F^2
 *            = (1/K) sum_k (||X_k||^2 - tr(G_k^+ Y_k^T X_k X_k^T Y_k)) / ||X_k||^2,  G_k = Y_k^T Y_k
 * (the paper draws Omega at random; training it is this library's extension).
 *
 * dpar2_sketch_loss_fwd: X, K, J, row_offsets (host, K + 1), ldx and dtype as
 *   for dpar2_compress; omega device J x l row-major FP32, 1 <= l <= min(J, 64).
 *   For 16-bit X, omega is rounded to X's type before use (as dpar2_compress
 *   rounds its test matrix).  Writes L to *loss (host) and keeps in the
 *   context what the backward pass needs (the sketch's QR factors, Q_k^T X_k,
 *   ||X_k||^2).  X must stay unchanged and valid until the matching backward.
 *   Slices whose sketch is rank deficient use the pseudo-inverse (the
 *   columns CholeskyQR2 drops).  Errors: INVALID_ARG / SHAPE before any launch.
 * dpar2_sketch_loss_bwd: grad_omega (device J x l FP32, caller-owned) <-
 *   grad_scale * dL/dOmega at the omega of the last forward on this context
 *   (for 16-bit X: at the rounded omega).  INVALID_ARG without a preceding
 *   successful forward.  Two more streams of X (four per training step). */
DPAR2_API dpar2_status dpar2_sketch_loss_fwd(dpar2_ctx* ctx, int K, int J, const int64_t* row_offsets, const void* X,
                                   int64_t ldx, dpar2_dtype dtype, const float* omega, int ell,
                                   double* loss, void* stream);
DPAR2_API dpar2_status dpar2_sketch_loss_bwd(dpar2_ctx* ctx, double grad_scale, float* grad_omega, void* stream);

/* In place: A (device rows x cols row-major FP32, 1 <= cols <= min(rows, 64))
 * <- A R^-1, an orthonormal basis of its column space by CholeskyQR2 (the QR
 * of Alg. 1's sketch; numerically dependent columns come out zero).  Used to
 * re-normalise a learned test matrix, whose loss depends on its column space
 * only.  Errors: INVALID_ARG (null A), SHAPE. */
DPAR2_API dpar2_status dpar2_orthonormalize(dpar2_ctx* ctx, int64_t rows, int cols, float* A, void* stream);

/* Post-fit analyses of the discovery section (Sec. IV-E).  The paper applies
 * them to the fitted factors of stock data: U_k of the stocks with a common
 * time range (equal I) and V's rows (latent feature vectors).
 *
 * dpar2_similarity: S(i, j) = exp(-gamma ||U_i - U_j||_F^2) (Eq. similarity)
 *   for K slices of one shape, each flattened to L = I R values: U device
 *   K x L row-major FP32 (row pitch ldu >= L floats; the U of dpar2_fit for
 *   K slices of equal length I is this layout with L = ldu = I R); S device
 *   K x K FP32 (row pitch lds >= K), written in full (symmetric, unit
 *   diagonal).  Squared distances come from the Gram matrix of the rows,
 *   n_i + n_j - 2 <U_i, U_j> (FP64 norms, Gram on the tensor cores with FP32
 *   accuracy: U split into three bf16 parts), clamped at zero.  Errors:
 *   INVALID_ARG / SHAPE before any launch, UNSUPPORTED without tensor maps.
 * dpar2_topk: for each of nrows rows of scores (device, row pitch ld >= n),
 *   the k largest values (1 <= k <= 16), largest first, equal values by
 *   lower column index, leaving out column exclude[row] (exclude: host,
 *   nrows ints, or NULL; -1 leaves nothing out): idx device nrows x k int32
 *   (-1 past the available columns), val device nrows x k FP32.  k-nearest
 *   neighbours: scores = rows of S, exclude = the targets.
 * dpar2_rwr: random walks with restarts on the similarity graph for nq
 *   queries at once (1 <= nq <= 16): adjacency A = S with a zero diagonal
 *   (no self loops), A~ = D^-1 A its row-normalised form (D the row sums;
 *   a zero row stays zero), r <- (1 - c) A~^T r + c q for `iters` steps from
 *   r = q, q one-hot at targets[query] (host, nq ints in [0, K)).  S device
 *   K x K symmetric (pitch lds), r device nq x K FP32 output.  The paper's
 *   settings are c = 0.15 and 100 steps.
 * dpar2_feature_pcc: C (device J x J FP32) <- the Pearson correlation
 *   coefficients between the rows of V (device J x R FP32, R >= 2); rows of
 *   zero variance give NaN. */
DPAR2_API dpar2_status dpar2_similarity(dpar2_ctx* ctx, int K, int64_t L, const float* U, int64_t ldu, double gamma,
                                        float* S, int64_t lds, void* stream);
DPAR2_API dpar2_status dpar2_topk(dpar2_ctx* ctx, int nrows, int n, const float* scores, int64_t ld,
                                  const int* exclude, int k, int* idx, float* val, void* stream);
DPAR2_API dpar2_status dpar2_rwr(dpar2_ctx* ctx, int K, const float* S, int64_t lds, int nq, const int* targets,
                                 double c, int iters, float* r, void* stream);
DPAR2_API dpar2_status dpar2_feature_pcc(dpar2_ctx* ctx, int J, int R, const float* V, float* C, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DPAR2_H_ */
