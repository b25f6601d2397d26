/*
 * tsqr.h -- C-ABI of the GB300 TSQR library (libtsqr.so).
 *
 * TSQR is the communication-avoiding Householder QR of a tall-skinny m x n matrix A (m >= n)
 * of Demmel, Grigori, Hoemmen and Langou, "Implementing Communication-Optimal Parallel and
 * Sequential QR Factorizations".  A is split into a 1-D block-row layout of leaves (Sec. 2,
 * Sec. 4.2).  Each leaf is factored by Householder QR; consecutive leaves owned by one thread
 * block are combined by the sequential flat-tree step QR([R; A_k]) (Algorithm 2); the R factors
 * of the thread blocks are then combined up an arity-q tree of structured QRs of stacked upper
 * triangles (Algorithm 1, Sec. 3.1 eq. fact_2rs).  The final R is the R of A; Q stays implicit
 * as the reified tree of Householder factors (Sec. 4.1) and is applied as Q^T B (a reduction)
 * or Q B (a broadcast), or expanded to the explicit thin Q (Sec. 7.2).
 *
 * Conventions shared by every call:
 *   - Matrices are FP64 (or FP32 with TSQR_F32), aligned to their element size, row-major:
 *     element (i, j) of X with leading dimension ldx is X[i * ldx + j] (ldx >= columns); or,
 *     with TSQR_COL_MAJOR, column-major: X[j * ldx + i] (ldx >= rows).  The layout given to
 *     tsqr_factor holds for that handle's R, Q and B too.  A is read by TMA, which needs a
 *     row-major A with a 16-byte aligned base and an even lda; any other A (column-major ones
 *     included, by a tiled transpose) is first copied into the workspace by a staging kernel.
 *   - Reflectors are H = I - tau v v^T with v_0 = 1; beta = -sign(alpha) ||x||, sign(0) = +1.
 *   - R is returned with a non-negative diagonal: D = diag(sign(R_jj)), R <- D R and the
 *     thin Q <- Q D (the QR is unique only up to these signs, Sec. 2).
 *   - The caller owns every buffer: A, R, B, Q and the workspace.  The library never allocates
 *     device memory; a handle is a small host object that points into the workspace, which
 *     must stay alive and untouched until tsqr_destroy.
 *   - Every call is stream-ordered and asynchronous on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream).  No call synchronises the host except tsqr_status_poll.
 *   - Errors are returned, never raised on the device: no device assert or trap.  Invalid
 *     shapes, strides or alignment return TSQR_ERR_INVALID_ARG before anything is launched.
 *     NaN and Inf in the input propagate to the outputs without being checked.
 *   - tsqr_last_error() gives a human-readable reason for the last failing call on the
 *     calling host thread.
 */
#ifndef TSQR_H_
#define TSQR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsqr_handle_s* tsqr_handle_t; /* opaque; owns no device memory */
typedef struct tsqr_batch_s* tsqr_batch_t;   /* opaque batch of factorizations; owns no device memory */
typedef void* tsqr_stream_t;                  /* a cudaStream_t */

typedef enum {
  TSQR_OK = 0,
  TSQR_ERR_INVALID_ARG = 1, /* bad shape, stride, pointer alignment or option */
  TSQR_ERR_UNSUPPORTED = 2, /* a valid request this build does not implement (e.g. n > 4096) */
  TSQR_ERR_CUDA = 3,        /* a CUDA runtime or driver call failed */
  TSQR_ERR_WORKSPACE = 4,   /* workspace missing or smaller than tsqr_workspace_size */
  TSQR_ERR_TIMEOUT = 5      /* a bounded device-side wait gave up (see tsqr_status_poll) */
} tsqr_status_t;

/* TSQR_F64: A, R, Q and B are binary64, arithmetic per tsqr_opts_t.precision.
 * TSQR_F32: A, R, Q and B are binary32 and every operation is binary32 (the FP32-level form of
 * the precision forms: backward error and loss of orthogonality of order n * 2^-24); for n in
 * 33..64 with leaf_h <= 128 the thin Q's Y M and, from 32 columns of B, Q^T B / Q B's Y^T B and
 * Y M run on the tensor cores as bf16x3 term products with FP32 accumulation.  A is widened
 * into the workspace first (it is never overwritten: inplace is not supported), and precision
 * must be 0.  Every call takes both; tsqr_backward then works in the same type. */
typedef enum { TSQR_F64 = 0, TSQR_F32 = 1 } tsqr_dtype_t;
/* TSQR_COL_MAJOR: n <= 64, not with inplace; tsqr_backward and batches take row-major only. */
typedef enum { TSQR_ROW_MAJOR = 0, TSQR_COL_MAJOR = 1 } tsqr_layout_t;

/* Tuning knobs of the reduction tree (Sec. 2: TSQR works on any tree; Sec. 4.2: the leaf
 * size follows from the fast-memory budget).  Zero means "choose automatically". */
typedef struct {
  int32_t leaf_h;    /* rows per leaf block: a multiple of 8, >= the padded n; 0 = auto */
  int32_t chain;     /* leaves combined sequentially by one thread block (flat tree);
                        1 = every leaf is its own tree leaf (pure arity-q tree); 0 = auto */
  int32_t arity;     /* children per node of the tree over thread blocks, 2..8; 0 = 2 */
  int32_t precision; /* 0 = native FP64 arithmetic everywhere.
                        1 = double-float: FP64 in and out, every operation of the path on pairs
                            of FP32 numbers (about 48 significant bits, unit roundoff ~2^-46) on
                            the FP32 pipe.  Magnitudes of A's and B's nonzero entries should lie
                            in about [2^-100, 2^100]; the stored factors (and A, with inplace)
                            then hold (hi, lo) FP32 pairs in each 8-byte slot.
                        2 = Ozaki WY: native FP64 reflectors, T recurrence and tree; the
                            compact-WY products of the thin Q (T C, Y M) and of Q^T B / Q B with
                            at least 32 columns of B (Y^T B, W^T T, Y M) as Ozaki splits (7
                            balanced base-256 digits in bf16, exact FP32 group sums) on the
                            tensor cores, and the flat-tree steps' Gram entries feeding T likewise
                            (n in 33..64, leaf_h <= 128; other shapes and narrower B run mode 0).
                            R and the reflectors are bitwise mode 0's.
                        3 = double-float factorization, and Q^T B / Q B with fewer than 32
                            columns; the tensor-core products as in mode 2 (other shapes run
                            mode 1).
                        With leaf_h = 64 at n in 33..64 and a binary tree, mode 2 factors by the
                        blocked step: FP64 reflectors per 16-column panel, the panel's WY
                        products and the Gram entries feeding T as Ozaki splits on the tensor
                        cores (FP32 storage likewise, with bf16x3 terms).
                        Batches factor mode 2 as 0 and mode 3 as 1, and form the thin Q of their
                        matrices of n in 33..64 (leaf_h <= 128) with the tensor-core products;
                        FP32-storage batches likewise with bf16x3 terms. */
  int32_t inplace;   /* nonzero: the leaf reflectors overwrite A (Sec. 4.2 storage) and A's
                        upper triangles hold intermediate R factors; zero: A is read only */
  int32_t r_only;    /* nonzero: compute R alone (the paper times R alone and Q with R apart,
                        Sec. 7): no reflectors, T or tree factors are stored or built, A is
                        read once and nothing else is written but R.  The handle then keeps no
                        Q: tsqr_apply_qt, tsqr_apply_q, tsqr_form_q and tsqr_backward return
                        TSQR_ERR_INVALID_ARG.  Not with inplace, n > 64 or a batch. */
} tsqr_opts_t;

/* Plan and storage of a factorization, for inspection and tests.  The pointers are device
 * pointers into the workspace (row-major FP64, np = n rounded up to a power of two >= 16).
 * For n > 64 (panels > 1) every field but m, n and panels describes the first panel's TSQR. */
typedef struct {
  int64_t m, n, np;
  int32_t leaf_h, chain, arity, depth; /* depth = levels of the tree above the chains */
  int64_t leaves, chains, tree_nodes;
  const double* v;        /* leaf reflectors, m x n with leading dimension ldv */
  int64_t ldv;
  const double* tau_leaf; /* leaves x np */
  const double* t_leaf;   /* leaves x np x np, upper triangular T of each leaf (Q = I - V T V^T) */
  const double* node_y;   /* tree_nodes x (arity-1) x np x np: the upper-triangular lower blocks
                             of each tree node's reflectors (their top block is I, eq. fact_2rs) */
  const double* node_tau; /* tree_nodes x np */
  const double* node_t;   /* tree_nodes x np x np */
  const double* signs;    /* np: D = diag(sign(R_jj)) of the root, sign(0) = +1 */
  int32_t panels;         /* 64-column panels of the factorization (1 when n <= 64) */
  int32_t dtype;          /* tsqr_dtype_t of A, R, Q and B */
  int32_t layout;         /* tsqr_layout_t of A, R, Q and B */
  const int32_t* status;  /* the device status word tsqr_status_poll reads (in the workspace;
                             bit 0: a bounded device wait gave up), so that tests can drive that
                             path from the host; the first panel's when panels > 1 */
} tsqr_info_t;

/* Bytes of device workspace tsqr_factor needs for an m x n factorization with `opts`
 * (NULL = all defaults).  Pure host computation. */
tsqr_status_t tsqr_workspace_size(tsqr_dtype_t dtype, int64_t m, int64_t n, const tsqr_opts_t* opts,
                                  size_t* bytes);

/* Factors A (m x n, m >= n >= 1, device, leading dimension lda >= n) into R and an implicit
 * Q (Algorithms 1 and 2, Sec. 3.1).  With inplace, lda must be even and A 16-byte aligned.
 * n <= 64 is one TSQR.  64 < n <= 4096 is a right-looking blocked QR over panels of 64 columns
 * (the panel factorization and trailing update of Sec. 6, Algorithm 3, on one GPU): panel p
 * (columns 64p.., rows 64p..m-1 of the updated matrix) is one TSQR, its Q^T updates the
 * trailing columns, and the top rows of that update are R's block row p.  A is then first
 * copied into the workspace, unless inplace is set, in which case A holds the updated matrix
 * and the panels' reflectors afterwards.
 *   dR     : device, n x n with ldr >= n; receives R with diag(R) >= 0, strict lower zeroed.
 *   dWork  : device workspace of at least tsqr_workspace_size bytes, 256-byte aligned.
 *   out    : receives a new handle (free with tsqr_destroy).  The handle records A's pointer
 *            when inplace is set; A must then outlive the handle.
 * A is read once from HBM; with inplace it is overwritten by the leaf reflectors. */
tsqr_status_t tsqr_factor(tsqr_dtype_t dtype, tsqr_layout_t layout, int64_t m, int64_t n, void* dA,
                          int64_t lda, void* dR, int64_t ldr, void* dWork, size_t work_bytes,
                          const tsqr_opts_t* opts, tsqr_stream_t stream, tsqr_handle_t* out);

/* B (m x k, device, ldb >= k) <- Q^T B with Q the full m x m orthogonal factor, signs
 * normalised (Sec. 4.1: applying Q^T is a reduction up the tree; Sec. 3.2 gives the node
 * update D = C0 + Y1^T C1, C0 -= T^T D, C1 -= Y1 T^T D).  Rows 0..n-1 of the result hold
 * Q_thin^T B; the other rows hold B's coordinates in this TSQR's orthogonal complement. */
tsqr_status_t tsqr_apply_qt(tsqr_handle_t h, int64_t k, void* dB, int64_t ldb, tsqr_stream_t stream);

/* B (m x k, device, ldb >= k) <- Q B with the same full Q (Sec. 4.1: a broadcast down the
 * tree).  tsqr_apply_q after tsqr_apply_qt returns B up to rounding. */
tsqr_status_t tsqr_apply_q(tsqr_handle_t h, int64_t k, void* dB, int64_t ldb, tsqr_stream_t stream);

/* Explicit thin Q (m x n, device, ldq >= n), signs normalised so that A = Q R (Sec. 2, the
 * thin factor; Sec. 7.2 counts this conversion in the Q-and-R runtime). */
tsqr_status_t tsqr_form_q(tsqr_handle_t h, void* dQ, int64_t ldq, tsqr_stream_t stream);

/* Synchronises `stream` and reads the handle's device status word: TSQR_OK, or
 * TSQR_ERR_TIMEOUT if any kernel of the handle's calls gave up a bounded wait. */
tsqr_status_t tsqr_status_poll(tsqr_handle_t h, tsqr_stream_t stream);

/* Fills *info with the plan and workspace pointers of h. */
tsqr_status_t tsqr_handle_info(tsqr_handle_t h, tsqr_info_t* info);

/* Reverse-mode derivative of (Q, R) = qr(A) through the handle's implicit Q.  Given the
 * cotangents Qbar = dL/dQ (m x n, device, ldqb >= n; NULL when L does not depend on Q) and
 * Rbar = dL/dR (n x n, device, ldrb >= n, upper triangle used: R's strict lower part is
 * structurally zero; NULL when L does not depend on R), writes
 * Abar = dL/dA (m x n, device, ldab >= n) by the published adjoint of the thin QR,
 *   M = R Rbar^T - Qbar^T Q,  Abar = (Qbar + Q copyltu(M)) R^{-T},  copyltu(M) = tril(M) + tril(M,-1)^T,
 * with Q^T Qbar and Q copyltu(M) applied from the implicit Q (tsqr_apply_qt, tsqr_apply_q):
 * no explicit Q is needed.  R (n x n, ldr >= n) is the R that tsqr_factor returned.  A must have
 * full column rank (the derivative does not exist otherwise; a zero R_jj gives Inf/NaN).  The
 * final solve keeps R in shared memory, so n > 154 (FP64) or n > 224 (FP32) returns
 * TSQR_ERR_UNSUPPORTED.  Every matrix has the factorization's dtype. */
tsqr_status_t tsqr_backward(tsqr_handle_t h, const void* dQbar, int64_t ldqb, const void* dRbar, int64_t ldrb,
                            const void* dR, int64_t ldr, void* dAbar, int64_t ldab, tsqr_stream_t stream);

/* ---- Batches: many independent tall-skinny factorizations in one launch --------------------
 * The s-step and block Krylov uses of TSQR (Sec. 1) produce many small tall-skinny blocks; a
 * batch factors all of them with one persistent launch of the factorization kernel (as many
 * blocks as fit on the GPU, each taking the next chain of any matrix from a work list ordered
 * longest chain first, until the list is used up) and forms their thin Q factors with one
 * launch per tree depth plus one chain launch.  All arrays below are host arrays of `count` entries; matrices
 * follow the conventions of tsqr_factor (A is read only; inplace is not supported).
 * tsqr_batch_factor and tsqr_batch_form_q only enqueue kernels and memsets on `stream`, so a
 * CUDA graph can capture them once and replay them; tsqr_batch_create plans the batch, uploads
 * its descriptors into the workspace and synchronises `stream` once. */
tsqr_status_t tsqr_batch_workspace_size(tsqr_dtype_t dtype, int32_t count, const int64_t* m, const int64_t* n,
                                        const tsqr_opts_t* opts, size_t* bytes);
/* dQ / ldq may be NULL (no thin Q); otherwise dQ[i] is m[i] x n[i] with ldq[i] >= n[i]. */
tsqr_status_t tsqr_batch_create(tsqr_dtype_t dtype, int32_t count, const int64_t* m, const int64_t* n,
                                void* const* dA, const int64_t* lda, void* const* dR, const int64_t* ldr,
                                void* const* dQ, const int64_t* ldq, void* dWork, size_t work_bytes,
                                const tsqr_opts_t* opts, tsqr_stream_t stream, tsqr_batch_t* out);
/* R of every matrix (Algorithms 1 and 2 per matrix). */
/* The same with a plan per matrix: item_opts holds `count` entries (leaf height, arity and chain
 * length of each matrix, e.g. an autotuner's choice for its shape; chain = 0 takes the batch's
 * shared chain length).  Every entry takes the same precision; TSQR_ERR_UNSUPPORTED otherwise.
 * The plans tune the tree to each shape (Sec. 7: the tuning space composes across levels). */
tsqr_status_t tsqr_batch_workspace_size_plans(tsqr_dtype_t dtype, int32_t count, const int64_t* m,
                                              const int64_t* n, const tsqr_opts_t* item_opts, size_t* bytes);
tsqr_status_t tsqr_batch_create_plans(tsqr_dtype_t dtype, int32_t count, const int64_t* m, const int64_t* n,
                                      void* const* dA, const int64_t* lda, void* const* dR, const int64_t* ldr,
                                      void* const* dQ, const int64_t* ldq, void* dWork, size_t work_bytes,
                                      const tsqr_opts_t* item_opts, tsqr_stream_t stream, tsqr_batch_t* out);
tsqr_status_t tsqr_batch_factor(tsqr_batch_t b, tsqr_stream_t stream);
/* Thin Q of every matrix (after tsqr_batch_factor). */
tsqr_status_t tsqr_batch_form_q(tsqr_batch_t b, tsqr_stream_t stream);
tsqr_status_t tsqr_batch_status_poll(tsqr_batch_t b, tsqr_stream_t stream);
tsqr_status_t tsqr_batch_destroy(tsqr_batch_t b);

/* R only, with no workspace and no allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc or hand the library a workspace: code inside
 * another runtime's allocator or its callbacks (which must not re-enter an allocator), plugins
 * whose host owns all device memory and gives them none, or C hosts without a device allocator.
 *   A  : device, m x n (m >= n >= 1), lda >= n and even, 16-byte aligned; read only.
 *   dR : device, n x n with ldr >= n; receives R with diag(R) >= 0, strict lower zeroed.
 * Same tree as tsqr_factor, except that the number of chains is capped so the scratch fits.
 * The scratch is a static 8 MiB device array inside libtsqr.so, held on every GPU that loads
 * the library until the process exits.  A problem whose tree needs more returns
 * TSQR_ERR_UNSUPPORTED.  The first call on a device looks up that array's address
 * (cudaGetSymbolAddress); make that first call before any stream capture starts.  Calls share
 * the array: each clears what must start at zero, and calls that overlap on the GPU (on
 * streams with no ordering between them) race and give wrong results.  The implicit Q is not
 * kept, so there is no handle.  The array's address is kept for the life of the process: do not
 * call this on a device after cudaDeviceReset.  If a device-side wait gives up (about one second
 * on a TMA copy; no fault, no trap), R is filled with NaN and the array's status word is set;
 * tsqr_noalloc_status_poll reports it. */
tsqr_status_t tsqr_factor_r_noalloc(int64_t m, int64_t n, const void* dA, int64_t lda, void* dR, int64_t ldr,
                                    tsqr_stream_t stream);
/* Outcome of the latest tsqr_factor_r_noalloc on the current device: waits for `stream` (the
 * stream that call used), then reads the static array's status word.  TSQR_OK, or
 * TSQR_ERR_TIMEOUT when a device-side wait gave up (R then holds NaN).  The next
 * tsqr_factor_r_noalloc clears the word.  If status_word is not NULL it receives the word's
 * device address (4 bytes; tests set it to check this path).  Allocates nothing. */
tsqr_status_t tsqr_noalloc_status_poll(tsqr_stream_t stream, void** status_word);

/* Frees the host handle (the workspace stays the caller's). NULL is a no-op. */
tsqr_status_t tsqr_destroy(tsqr_handle_t h);

const char* tsqr_status_string(tsqr_status_t s);
const char* tsqr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TSQR_H_ */
