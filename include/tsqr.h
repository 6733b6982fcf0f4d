/*
 * libtsqr -- the R factor of A = QR for tall-and-skinny matrices (m >> n) on one NVIDIA GB300
 * (sm_103a), computed TSQR-style after J. Langou, "Computing the R of the QR factorization of
 * tall and skinny matrices using MPI_Reduce" (arXiv:1002.4250):
 *   step 1 (Section 2, Section 3 / Table 1): every row tile of A gets a local Householder QR;
 *   step 2 (Section 2, Table 3): the tiles' n x n upper-triangular factors are reduced along a
 *          tree by the operator qr(R_i, R_j) = R factor of [R_i; R_j], which does no arithmetic
 *          on the known zeros of the two triangles.
 * The tree is fixed per call (binary, flat or hybrid; Section 1 and Fig. 1), so a call is
 * bit-reproducible: same inputs and same plan give the same bytes.  Wide tall matrices (and,
 * through tsqr_caqr_r, any width) run by panels of columns, each a reduction of its own
 * followed by an update of the columns right of it (Section 5).
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major: element (i, j) of A is A[i + j*lda].
 *   - R is n x n, written in full: the upper triangle with diag(R) >= 0 (Section 2: R is unique
 *     up to the sign of each row; a non-negative diagonal makes it unique) and an exact zero
 *     strict lower triangle.  R is always FP64.
 *   - Pointers named "device" must be device (or managed) memory of the current device; the
 *     caller owns every buffer; the library never frees or keeps caller memory.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy default stream).
 *     Argument errors are found on the host and returned before anything is enqueued.
 *     Conditions met on the device (non-finite values in R) are recorded in a per-stream
 *     status word that tsqr_get_device_status() reads.
 *   - Workspace (tree-node slots and counters) is allocated by the library, per device and
 *     stream, with stream-ordered allocation, grown when needed and reused across calls;
 *     tsqr_release_workspace() returns it.  Calls on the same stream may follow each other
 *     freely; the first call on a stream should not be made under stream capture.  A few
 *     calls also allocate a buffer for the call itself, stream-ordered, as each one states.
 *   - n is limited to TSQR_MAX_N except where a call says otherwise (the FP64 R calls by
 *     panels, tsqr_caqr_r and tsqr_lstsq take any n <= m).
 */
#ifndef LIBTSQR_TSQR_H
#define LIBTSQR_TSQR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSQR_MAX_N 128

typedef enum {
    TSQR_SUCCESS = 0,
    TSQR_ERR_INVALID_ARG = 1,   /* a size, leading dimension, pointer or enum is invalid      */
    TSQR_ERR_UNSUPPORTED = 2,   /* valid but not supported (e.g. n > TSQR_MAX_N)              */
    TSQR_ERR_CUDA = 3,          /* a CUDA runtime call failed (launch, allocation, copy)      */
    TSQR_ERR_ALLOC = 4,         /* workspace could not be allocated                           */
    TSQR_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up (read by
                                   tsqr_get_device_status)                                    */
    TSQR_STATUS_NONFINITE = 6   /* R holds NaN or Inf (the input held NaN/Inf or overflowed)  */
} tsqr_status_t;

/* Storage type of A.  R is always FP64. */
typedef enum { TSQR_F64 = 0, TSQR_F32 = 1, TSQR_BF16 = 2 } tsqr_dtype_t;

/* Arithmetic of the leaf (tile) factorizations.  The tree operator is FP64 in every mode.
 * TSQR_PREC_F64:   FP64 everywhere (A must be TSQR_F64).
 * TSQR_PREC_MIXED: leaf Householder panels in FP32 (A is FP32 or BF16, widened exactly on
 *                  load); the reflector scalars and the leaf's R in FP64 (FOLD leaf) or
 *                  double-FP32, about 48 bits (PANELS leaf); tree combines in FP64.          */
typedef enum { TSQR_PREC_F64 = 0, TSQR_PREC_MIXED = 1 } tsqr_prec_t;

/* Reduction tree over the row tiles (Section 1: "any reduction tree" works by associativity).
 * BINARY: one tile of tile_rows rows per leaf, leaves paired (2t, 2t+1) level by level, the
 *         lower index on top, an odd last node promoted unchanged (Fig. 1 for four leaves).
 * FLAT:   one CTA folds every tile in row order, R <- R([R; A_t]) (the tile algorithms' tree).
 * HYBRID: `ctas` CTAs each fold a contiguous run of tiles flat, their R factors then reduced
 *         by a fixed tree of `arity` children per node (children in index order, the lowest on
 *         top; a lone last child promoted unchanged).
 * PANELS: FP64 R only (tsqr_r, tsqr_r_ex with F64/F64): the columns in panels of `tile_rows`
 *         columns (0 = 16), each panel's R by its own TSQR reduction (AUTO plan, reflectors
 *         kept) and its Q^T applied to the columns right of it, as tsqr_caqr_r does (Section
 *         5's panel and update).  R equals one reduction's up to rounding.
 * AUTO picks HYBRID, or PANELS for FP64 R with n >= 56 and m >= 8 n, where it measured faster
 * (4,194,304 rows, n = 56 / 64 / 96 / 128: 775 / 828 / 863 / 887 against 727 / 750 / 555 / 586
 * GFLOP/s; at n = 48 one reduction is faster, 826 against 802).                           */
typedef enum {
    TSQR_TREE_AUTO = 0, TSQR_TREE_BINARY = 1, TSQR_TREE_FLAT = 2, TSQR_TREE_HYBRID = 3,
    TSQR_TREE_PANELS = 4
} tsqr_tree_t;

/* Leaf (tile) factorization of the MIXED path (TSQR_PREC_MIXED; the FP64 path has one leaf).
 * FOLD:   the fused fold R <- R([R; chunk]) one reflector at a time, every reflector applied to
 *         every later column by the CUDA cores (FP32 bulk arithmetic, FP64 R and scalars); any
 *         n <= TSQR_MAX_N.
 * PANELS: the same fold by panels of 16 columns: each panel factorized column by column in
 *         registers (FP32 dot products; the reflector scalars in double-FP32, about 48 bits),
 *         then applied to the columns right of it as one compact WY block (I - V S V^T) whose
 *         two products run on the tensor cores as split-TF32 products with FP32 accumulation
 *         (each as accurate as an FP32 dot product); R in double-FP32 in the leaf, FP64 in the
 *         tree.  n <= 112; chunks of 256, 384, 512, 640, 768 or 1024 rows (tile_rows; AUTO:
 *         the tallest the width's shared and tensor memory allow).
 * AUTO picks PANELS for n <= 112 (FP32 from n = 9, BF16 from n = 3), where it measured
 * faster, else FOLD. */
typedef enum { TSQR_LEAF_AUTO = 0, TSQR_LEAF_FOLD = 1, TSQR_LEAF_PANELS = 2 } tsqr_leaf_t;

/* Optional plan override.  Zero fields mean "choose".  The chosen plan fixes the arithmetic
 * order, so two calls with equal plans and inputs return identical bytes. */
typedef struct {
    int32_t tree;       /* tsqr_tree_t                                                     */
    int32_t tile_rows;  /* rows per tile (slab) b; must fit the kernel's shared memory      */
    int32_t ctas;       /* HYBRID: number of leaf CTAs                                      */
    int32_t warps;      /* bulk warps per CTA (1 .. 12)                                      */
    int32_t arity;      /* children per tree node, 2..8.  BINARY uses 2, the operator of
                           Table 3; a node with c > 2 children folds their c stacked triangles
                           in one sweep (the R factor of [R_1; ...; R_c], equal to a sequence of
                           binary operators by associativity, Section 2).  0 = as many as the
                           kernel's shared memory holds.                                     */
    int32_t leaf;       /* tsqr_leaf_t (mixed path only; 0 elsewhere).  With PANELS,
                           tile_rows is the chunk height (256, 384, 512, 640, 768 or 1024) of a HYBRID
                           plan, warps is 8 (or 0).                                          */
} tsqr_plan_t;

typedef void *tsqr_stream_t; /* a cudaStream_t */

/* R factor of the m x n FP64 matrix A (Section 2, steps 1 and 2).
 *   A   : device, column-major, lda >= max(1, m); read only.
 *   m   : rows, m >= 0 (m = 0 gives R = 0; m < n gives rows m..n-1 of R equal to zero).
 *   n   : columns, 0 <= n <= TSQR_MAX_N (n = 0 does nothing); above TSQR_MAX_N, any n <= m,
 *         by panels (the PANELS tree, as tsqr_caqr_r), else TSQR_ERR_UNSUPPORTED.
 *   R   : device, column-major n x n, ldr >= max(1, n); fully written.
 * Uses the AUTO plan.  Returns TSQR_SUCCESS once the work is enqueued.                     */
tsqr_status_t tsqr_r(const double *A, int64_t m, int64_t n, int64_t lda, double *R, int64_t ldr,
                     tsqr_stream_t stream);

/* tsqr_r for A and R in HOST memory, FP64.  TSQR needs no copy of A before it starts (Section 2:
 * each row block is factorized on its own and only the n x n factors meet in the tree), so
 * page-locked A (cudaHostAlloc / cudaHostRegister with a device mapping) is read IN PLACE by
 * tsqr_r's kernel through its device address: every leaf streams its rows from host memory
 * while it factorizes them, with no second stream, flag or wait, so the result does not
 * depend on copies and kernels running at the same time.  Plan, kernel and R are tsqr_r's, bit
 * for bit.  Other host memory (pageable) is copied whole to a device buffer of the workspace
 * first.  Where the AUTO plan runs by panels (n >= 56, m >= 8 n), A is copied whole to a buffer
 * of the call (stream-ordered) and the panels run on it, as tsqr_r does (R equals tsqr_r's bytes).
 *   A : host, column-major m x n, lda >= m.
 *   R : host, column-major n x n, ldr >= n, written as by tsqr_r.
 * Asynchronous on `stream` like tsqr_r: A must not be modified, nor R read, until the stream
 * has been synchronized (for m = 0, R is zeroed before the call returns).  Workspace: the tree's
 * slots and R, plus A's size when A is copied, from the per-stream pool. */
tsqr_status_t tsqr_r_host(const double *A, int64_t m, int64_t n, int64_t lda, double *R,
                          int64_t ldr, tsqr_stream_t stream);

/* tsqr_r (Section 2, steps 1 and 2) with the storage type of A, the leaf arithmetic and an
 * optional plan (NULL = AUTO): the plan fixes the tree (Section 1: any reduction tree works),
 * the tile rows, the leaves, the bulk warps and the arity.
 * (dtype, prec) must be (F64, F64), (F32, MIXED) or (BF16, MIXED).  lda counts elements.
 * MIXED keeps A in its storage type on chip and does the leaves' bulk arithmetic in FP32,
 * with the reflector scalars and the leaf's R in FP64 (FOLD leaf) or double-FP32 (PANELS leaf,
 * see tsqr_leaf_t) and the tree in FP64; R is always FP64. */
tsqr_status_t tsqr_r_ex(const void *A, int32_t dtype, int32_t prec, int64_t m, int64_t n,
                        int64_t lda, double *R, int64_t ldr, const tsqr_plan_t *plan,
                        tsqr_stream_t stream);

/* One node of the reduction tree on the GPU: the operator qr(R1, R2) of Section 2 / Table 3,
 * the R factor of the 2n x n stack [R1; R2] of two upper triangles (entries below their
 * diagonals are ignored), computed with the same reflector sign rule as the tree
 * (beta = -sign(alpha) ||.||, sign(0) = +1).
 *   R1, R2 : device, column-major n x n, ld1, ld2 >= n; read only.
 *   R      : device, column-major n x n, ldr >= n: the R factor, strict lower part zero;
 *            with normalize != 0 rows are also flipped so that diag(R) >= 0.             */
tsqr_status_t tsqr_qr_uppers(int64_t n, const double *R1, int64_t ld1, const double *R2,
                             int64_t ld2, double *R, int64_t ldr, int32_t normalize,
                             tsqr_stream_t stream);

/* Thin QR: Q (m x n, orthonormal columns) and R (n x n, diag(R) >= 0) with A = Q R, FP64.
 * Section 3 notes that the Q factor is obtained by applying the Householder transformations
 * of the reduction to the identity, which requires keeping every node's Householder vectors
 * and the shape of the tree.  This call does that: the factorization is tsqr_r's (same plan,
 * same kernels, the same R bit for bit; with the AUTO plan, except at widths where tsqr_r's
 * plan runs a number of bulk warps other than 4, 8 or 12, or chunks too tall for the Q passes'
 * buffers, which take the four-warp plan instead: tsqr_last_plan reports the plan used) with
 * the reflectors of every leaf chunk and tree node
 * kept, then Q = H [I_n; 0] (with the sign convention applied to Q's columns) is formed top-down
 * through the tree and backwards through each leaf's chunks.  Q is unique for A of full rank
 * (as R is); with Householder reflectors it is then orthonormal to working accuracy however
 * ill-conditioned A is.  For rank-deficient A (a zero on R's diagonal) A = Q R still holds,
 * but the columns of Q beyond the rank are not guaranteed orthonormal: each leaf's first chunk
 * is folded under a zero triangle, and the part of Q that an identity reflector leaves in
 * those rows is dropped (the zero matrix gives Q = 0).
 *   A    : device, column-major m x n, lda >= m; read only.  m >= n >= 1.
 *   Q    : device, column-major m x n, ldq >= m; must not overlap A.  It also serves as the
 *          store of the leaf reflectors between the two passes.
 *   R    : device, column-major n x n, ldr >= n.
 *   plan : NULL = AUTO, or as for tsqr_r_ex with warps 0, 4, 8 or 12 (other counts return
 *          TSQR_ERR_INVALID_ARG).  The plan's chunking must put every chunk boundary at a
 *          multiple of its chunk height (AUTO and HYBRID/FLAT plans do; a BINARY tile taller
 *          than one chunk that is not a multiple of it does not).
 * Every n <= TSQR_MAX_N is supported: where a chunk of tails, the Q rows and the carried block
 * do not fit shared memory together (n above about 64 with the AUTO plan), the passes take Q's
 * columns in groups and the tails go to workspace instead of Q.  Workspace: about (2 + arity)
 * n^2 doubles per tree node plus 2n per chunk, plus m x n when grouped, from the per-stream
 * pool.  Launches: the factorization, one per tree level below the root, and one leaf pass per
 * column group. */
tsqr_status_t tsqr_qr(const double *A, int64_t m, int64_t n, int64_t lda, double *Q,
                      int64_t ldq, double *R, int64_t ldr, const tsqr_plan_t *plan,
                      tsqr_stream_t stream);

/* Least squares: X minimizing ||A X - B||_F column by column, for A of full column rank, FP64.
 * Section 3 notes that the reduction's Householder transformations, once stored, can be applied
 * to another matrix (there: the trailing matrix of a blocked QR).  This call applies Q^T to B:
 * the factorization is tsqr_qr's with the reflectors kept; each leaf folds its rows of B into the n rows of Q^T B that belong to its R
 * and the tree combines them with the stored node reflectors; then R X = (Q^T B)(0:n, :).  Q is
 * never formed.
 *   A : device, column-major m x n, lda >= m, m >= n >= 1; read only.
 *   B : device, column-major m x k, ldb >= m, k >= 0; read only.
 *   X : device, column-major n x k, ldx >= n.
 *   R : device n x n (ldr >= n) receiving R, or NULL.
 *   plan as for tsqr_qr (NULL = AUTO).
 * With few right-hand sides (k <= max(1, n / 4) and n + k <= TSQR_MAX_N) the augmented matrix
 * [A | B] is factorized instead (its R holds R and (Q^T B)(0:n, :) side by side) and one
 * triangular solve follows; R then equals tsqr_r's up to rounding.  Otherwise the columns of B
 * go k_g = min(k, n) at a time (two launches per group after the factorization) and R is
 * tsqr_qr's bit for bit (tsqr_r's under the plan tsqr_last_plan reports).
 * Above TSQR_MAX_N columns (AUTO plan only) [A | B] is copied to a buffer allocated for the
 * call (stream-ordered, m (n + k) doubles, plus (n + k)^2 for its R) and factorized by panels
 * as tsqr_caqr_r does; its R holds R and (Q^T B)(0:n, :) side by side, then one triangular
 * solve.  R then equals tsqr_caqr_r's on A up to rounding.
 * A zero on R's diagonal (rank deficiency) makes X non-finite and the device status
 * TSQR_STATUS_NONFINITE.  Returns TSQR_ERR_UNSUPPORTED where tsqr_qr does (n <= TSQR_MAX_N), or
 * for an explicit plan above TSQR_MAX_N columns. */
tsqr_status_t tsqr_lstsq(const double *A, int64_t m, int64_t n, int64_t lda, const double *B,
                         int64_t ldb, int64_t k, double *X, int64_t ldx, double *R, int64_t ldr,
                         const tsqr_plan_t *plan, tsqr_stream_t stream);

/* R of a general tall m x n matrix (n not limited to TSQR_MAX_N), FP64, by the communication-
 * avoiding QR that Section 5 describes: the first `panel` columns (the panel) are factorized by
 * the TSQR reduction with their Householder reflectors kept, Q^T of that panel is applied to
 * the columns right of it (its first `panel` rows are R's next block row), and the rows left
 * below form the next panel's matrix; and so on to the last column.
 *   A     : device, column-major m x n, lda >= m, m >= n >= 1; read only.
 *   R     : device, column-major n x n, ldr >= n; the upper triangle with diag(R) >= 0, the
 *           strict lower triangle written as 0.  Must not overlap A.
 *   panel : panel width, 1 .. TSQR_MAX_N; 0 = 16 (or n if smaller).
 *   plan  : NULL = AUTO, else the plan used for every panel's factorization (as for tsqr_qr).
 * Each panel's update keeps every row of the panel's matrix and adds the n-row blocks its tree
 * nodes leave behind: a panel factorized on L leaves adds (L - 1) panel rows to the next
 * matrix (the rows' order does not change R).  Workspace: the matrix right of the first panel
 * with those rows added (about 8 (m + (n / panel) (L - 1) panel) n bytes), the panel's stored
 * reflectors (8 m panel bytes) and small tree buffers, from the per-stream pool.  Launches:
 * three per panel (the factorization, its chunks' compact WY factors and the update; two where
 * the blocked update does not fit) except the last (the factorization alone).  Returns
 * TSQR_ERR_INVALID_ARG for bad sizes, TSQR_ERR_UNSUPPORTED for a panel above TSQR_MAX_N or a
 * plan tsqr_qr would refuse, TSQR_ERR_ALLOC when the workspace cannot be had. */
tsqr_status_t tsqr_caqr_r(const double *A, int64_t m, int64_t n, int64_t lda, double *R,
                          int64_t ldr, int64_t panel, const tsqr_plan_t *plan,
                          tsqr_stream_t stream);

/* Varlen batch of independent problems: R_i = R factor of A_i for i < count, each the TSQR of
 * Section 2 (steps 1 and 2) with its own leaves and tree, all in one persistent launch.
 *   ptrs    : host array of `count` device pointers; A_i is column-major m_i x n_i with
 *             lda_i = m_i (e.g. all pointing into one packed buffer).
 *   ms, ns  : host arrays of count rows (>= 0) and columns (1..TSQR_MAX_N).
 *   offsets : host array of count+1 non-decreasing element offsets into R_packed with
 *             offsets[i+1] - offsets[i] >= n_i^2; R_i is written column-major with ld n_i at
 *             R_packed + offsets[i].
 *   R_packed: device FP64 buffer of at least offsets[count] elements.
 *   dtype, prec as for tsqr_r_ex.  All problems are factorized by one launch: FP64 and wider
 *   mixed batches by the fold leaf, mixed batches up to 112 columns by the blocked
 *   tensor-core leaf of TSQR_LEAF_PANELS (see tsqr_batch_plan_t's leaf).                    */
tsqr_status_t tsqr_r_batched(const void *const *ptrs, const int64_t *ms, const int32_t *ns,
                             const int64_t *offsets, int32_t count, double *R_packed,
                             int32_t dtype, int32_t prec, tsqr_stream_t stream);

/* Knobs of a varlen batch call: the leaf and tree choices of Section 2 made once per batch
 * (the paper factorizes one matrix; a batch has many).  A field of 0 takes the library's rule.
 *   warps          : bulk warps per CTA, 1 .. 12 (0: 12 for a batch with widths from 48 on
 *                    whose widest chunk fits with 12 warps, else 4).
 *   ctas_per_sm    : chunk height: 1 = chunks as tall as fit one CTA per SM, 2 = as fit two
 *                    (0: 2 when the widest problem's chunk still holds two rows per lane).
 *                    The grid is as many CTAs per SM as the occupancy allows.
 *   leaves_per_cta : leaf size: a leaf holds about (sum of max(m_i, 1) n_i^2) / (CTAs x
 *                    leaves_per_cta) of work, in whole chunks; 1 .. 64 (0: 6).
 *   arity[b]       : tree arity of the problems in width bucket b (n <= 8, <= 16, <= 32,
 *                    > 32), 2 .. 8, lowered to what the width's shared memory holds (0: the
 *                    largest that fits).
 *   leaf           : mixed precision only, a tsqr_leaf_t: FOLD, or PANELS (the blocked
 *                    tensor-core leaf of tsqr_r_ex, for batches up to 112 columns; chunks as
 *                    tall as the widest problem allows, 8 warps, one CTA per SM, so warps and
 *                    ctas_per_sm do not apply).  0: PANELS up to 112 columns, else FOLD.
 *                    PANELS for an FP64 batch or one wider than 112 columns returns
 *                    TSQR_ERR_UNSUPPORTED. */
typedef struct tsqr_batch_plan_t {
    int32_t warps;
    int32_t ctas_per_sm;
    int32_t leaves_per_cta;
    int32_t arity[4];
    int32_t leaf;
} tsqr_batch_plan_t;

/* tsqr_r_batched with explicit knobs.  plan: NULL or all zero = AUTO (the batch's tuned plan
 * if tsqr_autotune_batched tuned its shape bucket on this device, else the built-in rules).
 * Returns TSQR_ERR_INVALID_ARG for a field out of its range, TSQR_ERR_UNSUPPORTED when the
 * widest problem's chunk does not fit the requested warps and chunk height. */
tsqr_status_t tsqr_r_batched_ex(const void *const *ptrs, const int64_t *ms, const int32_t *ns,
                                const int64_t *offsets, int32_t count, double *R_packed,
                                int32_t dtype, int32_t prec, const tsqr_batch_plan_t *plan,
                                tsqr_stream_t stream);

/* Batch autotuning: times knob settings on the caller's batch and caches the fastest for its
 * shape bucket: the device, the input type, the set of width buckets present, floor(log2
 * count) and floor(log2 of the work sum max(m_i, 1) n_i^2).  From then on an AUTO batched call
 * (tsqr_r_batched, or tsqr_r_batched_ex with plan NULL or all zero) in that bucket uses it and
 * returns the bytes it gives.  The search starts from the built-in rules and moves one knob at a
 * time: for a mixed batch up to 112 columns the fold leaf against the blocked one, then (for
 * the fold) warps (4, 6, 8, 12) x ctas_per_sm, then leaves_per_cta, then each present width bucket's arity
 * (2, 4, 8); each setting is run once to warm up and timed over one call with CUDA events on
 * `stream`.
 *   Arguments as for tsqr_r_batched; R_packed is overwritten.  best: optional, receives the
 *   chosen knobs.  Synchronizes `stream`; not for use under stream capture.  Returns
 *   TSQR_ERR_INVALID_ARG for count == 0. */
tsqr_status_t tsqr_autotune_batched(const void *const *ptrs, const int64_t *ms, const int32_t *ns,
                                    const int64_t *offsets, int32_t count, double *R_packed,
                                    int32_t dtype, int32_t prec, tsqr_batch_plan_t *best,
                                    tsqr_stream_t stream);

/* The knobs the last batched call (tsqr_r_batched, tsqr_r_batched_ex) on this host thread ran
 * with: warps, ctas_per_sm, leaves_per_cta and leaf as resolved, arity as given (0 = the
 * largest that fits).  All zero before any batched call and after one that launched nothing.
 *   out : host pointer, required.  Returns TSQR_ERR_INVALID_ARG when NULL. */
tsqr_status_t tsqr_last_batch_plan(tsqr_batch_plan_t *out);

/* Size of the fixed device array tsqr_r_noalloc works in (16 MiB). */
#define TSQR_NOALLOC_SCRATCH_BYTES (16u << 20)

/* tsqr_r for callers that cannot allocate device memory when they call: for example a serving
 * loop that must not allocate after start-up, or a process whose framework has already
 * reserved the device's memory for its own caching allocator.  The paper has no counterpart;
 * this is a deployment variant of tsqr_r.
 *   Same arguments as tsqr_r (FP64).  It always runs ONE reduction with the AUTO plan's
 *   one-reduction partition (tsqr_resolve_plan's plan, or the tuned plan of the bucket): where
 *   tsqr_r's AUTO plan runs by panels (n >= 56, m >= 8 n), this call does not, and its R equals
 *   tsqr_r's within the parity tolerance, not bit for bit; elsewhere the plan, kernel and R are
 *   tsqr_r's.  Instead of the per-stream workspace it uses one static device array of
 *   TSQR_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the process
 *   exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     and keeps it for the life of the process; make that first call before any stream capture
 *     on that device.  The address does not survive cudaDeviceReset: do not call this
 *     function on a device after resetting it.
 *   - All calls share the array and it keeps the last call's contents (each call clears the
 *     part that must start at zero): calls that overlap on the GPU, on any streams, race and
 *     must be serialized by the caller.
 *   - A problem whose reduction tree needs more than the array (one n x n FP64 slot and one
 *     counter per tree node; with the AUTO plan every n <= 80 fits, n = 128 does not)
 *     returns TSQR_ERR_UNSUPPORTED before enqueuing anything.
 *   - No device status is recorded: NaN/Inf still propagate into R, but
 *     tsqr_get_device_status() does not report them for these calls.
 *   - tsqr_last_plan and tsqr_last_launch_count describe the call like any other.           */
tsqr_status_t tsqr_r_noalloc(const double *A, int64_t m, int64_t n, int64_t lda, double *R,
                             int64_t ldr, tsqr_stream_t stream);

/* Plan autotuning: times candidate plans for an (m, n, dtype, prec) problem on the caller's A
 * and caches the fastest.  From then on every AUTO call (plan NULL or all fields zero: tsqr_r,
 * tsqr_r_ex, tsqr_qr, tsqr_r_noalloc, tsqr_resolve_plan) on the same device with the same n,
 * the same leaf precision and the same floor(log2 m) uses the tuned plan, and returns the
 * bytes that plan gives.  The paper has no counterpart: its trees are picked by hand or by the
 * MPI library (Section 1).
 *   A, m, n, lda, dtype, prec, R, ldr as for tsqr_r_ex; R is overwritten (the last candidate's
 *   result).  best: optional, receives the chosen plan.
 *   Candidates: HYBRID slabs as tall as fit 1, 2 or 3 CTAs per SM, and half as tall, with that
 *   many CTAs per SM on every SM; 4, 5, 6, 8 or 12 bulk warps; for FP64 from n = 48 (m >= 8 n) the
 *   PANELS tree with 16- and 32-column panels; for the mixed path up to n = 112 the blocked
 *   leaf with every chunk height (256 to 1024 rows) the width's shared and tensor memory hold,
 *   1 to as many CTAs per SM as fit.  Then the fastest HYBRID plan with tree arity 2, 3, 4, 6
 *   and 8.  Each is timed over three calls with CUDA events on `stream`.
 *   Synchronizes `stream`; not for use under stream capture.  Returns TSQR_ERR_UNSUPPORTED if
 *   no candidate runs. */
tsqr_status_t tsqr_autotune(const void *A, int32_t dtype, int32_t prec, int64_t m, int64_t n,
                            int64_t lda, double *R, int64_t ldr, tsqr_plan_t *best,
                            tsqr_stream_t stream);

/* Forgets every tuned plan, single-matrix and batched: AUTO calls go back to the built-in
 * rules. */
void tsqr_autotune_reset(void);

/* Synchronizes `stream`, returns the device-side status recorded by the calls made on it since
 * the last query (TSQR_SUCCESS or TSQR_STATUS_NONFINITE) and clears it.  TSQR_ERR_CUDA if the
 * stream reports an error. */
tsqr_status_t tsqr_get_device_status(tsqr_stream_t stream);

/* Frees every workspace the library holds (all devices and streams) after synchronizing
 * the devices it used.  Safe to call at any time no call is in flight. */
void tsqr_release_workspace(void);

/* Static description of a status code. */
const char *tsqr_status_string(int32_t status);

/* The plan of the factorization the last call on this host thread ran (the first panel's for
 * tsqr_caqr_r), in the form tsqr_r_ex accepts: passed back as a plan it gives the same
 * partition, kernels and bytes.  All fields zero when that call ran no factorization.
 *   out : host pointer, required.  Returns TSQR_ERR_INVALID_ARG when NULL. */
tsqr_status_t tsqr_last_plan(tsqr_plan_t *out);

/* The plan AUTO (or `plan`) resolves to for an (m, n, dtype, prec) problem on the current
 * device, written to *out.  Host only; enqueues nothing. */
tsqr_status_t tsqr_resolve_plan(int64_t m, int64_t n, int32_t dtype, int32_t prec,
                                const tsqr_plan_t *plan, tsqr_plan_t *out);

/* Number of kernel launches the last successful call on this host thread enqueued. */
int32_t tsqr_last_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* LIBTSQR_TSQR_H */
