/*
 * figaro.h -- C ABI of the GB300 FiGaRo library.
 *
 * FiGaRo (Olteanu, Vortmeier, Zivanovic, "Givens Rotations for QR Decomposition, SVD
 * and PCA over Database Joins", arXiv 2204.00525) computes the upper-triangular R of
 * the QR decomposition of A[:, Y], the data columns of the natural join of an acyclic
 * database, without materialising the join (§2 "Input"/"Output", Theorem of §6), and
 * from R the SVD and PCA of A (§8.2-8.3).  Every step runs in CUDA kernels on one
 * GPU; the host code only validates, plans and launches.
 *
 * Conventions shared by every entry point
 *   - Status: every function returns an int, FIGARO_OK (0) on success, else one of
 *     figaro_status.  figaro_error_string() names a status; figaro_last_error()
 *     returns a message with details about the most recent failure of this thread.
 *   - Memory: in FIGARO_MEM_DEVICE mode (the default) every data pointer (key columns,
 *     data, R, sigma, V, components, eigvals) is a device pointer of the current CUDA
 *     device; in FIGARO_MEM_HOST mode they are host pointers (pinned memory gives
 *     asynchronous copies) and the library copies inputs in and results out on the
 *     plan's stream.  The caller owns all input and output buffers; inputs must stay
 *     valid and unchanged while a call that reads them is running.  The plan owns its
 *     device workspace and frees it in figaro_plan_destroy.
 *   - Streams: all device work is enqueued on the stream given to figaro_plan (a
 *     cudaStream_t passed as void*, NULL for the legacy default stream).  The compute
 *     calls block the calling host thread only at their end, to read one device error
 *     word; they may be called again on the same plan once they have returned.
 *   - Column order of A[:, Y], R, V and the components: relation order 0..n_rel-1,
 *     then data-column order inside each relation (the [T_1 ... T_r] layout of Alg. 4).
 *   - Threads: a plan must not be used by two host threads at once.
 */
#ifndef FIGARO_H
#define FIGARO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum figaro_status {
  FIGARO_OK = 0,
  FIGARO_ERR_INVALID_ARG = 1,   /* a null pointer, negative size, bad enum, ld too small  */
  FIGARO_ERR_INVALID_TREE = 2,  /* parent[] is not a tree, or it is not a join tree (§2:
                                   the relations holding an attribute must be connected),
                                   or a key attribute occurs in a single relation         */
  FIGARO_ERR_NOT_REDUCED = 3,   /* require_reduced was set and a tuple does not join     */
  FIGARO_ERR_OVERFLOW = 4,      /* a join count (§5) exceeds 2^64 - 1 (unsigned 64 bits)  */
  FIGARO_ERR_NOMEM = 5,         /* device or host allocation failed                      */
  FIGARO_ERR_TIMEOUT = 6,       /* an iteration limit was reached (Jacobi sweeps)         */
  FIGARO_ERR_CUDA = 7,          /* a CUDA runtime call failed (see figaro_last_error)     */
  FIGARO_ERR_KEY_RANGE = 8,     /* a key value lies outside the range seen by figaro_plan */
  FIGARO_ERR_NOT_SORTED = 9,    /* presorted was set but a relation is not sorted         */
  FIGARO_ERR_UNSUPPORTED = 10,  /* a size limit of this build (see below) is exceeded     */
  FIGARO_ERR_SINGULAR = 11      /* figaro_backward: R has a zero diagonal entry           */
};

enum { FIGARO_KEY_I64 = 0, FIGARO_KEY_I32 = 1 };
enum { FIGARO_COL_MAJOR = 0, FIGARO_ROW_MAJOR = 1 };
enum { FIGARO_PREC_FP64 = 0, FIGARO_PREC_MIXED = 1, FIGARO_PREC_MIXED_REFINED = 2 };
enum { FIGARO_LEAF_HOUSEHOLDER = 0, FIGARO_LEAF_GIVENS = 1, FIGARO_LEAF_TCGEN05 = 2, FIGARO_LEAF_MMA_SYNC = 3 };
enum { FIGARO_MEM_DEVICE = 0, FIGARO_MEM_HOST = 1 };

/* One relation S_i (§2 "Relations and Joins").
 *   n_rows    M_i >= 1, at most 2^31 - 1.
 *   n_keys    number of key (join) attributes K_i (0 allowed: a relation joined by
 *             Cartesian product).  At most 8.
 *   key_attr  host array [n_keys]: global attribute id (>= 0) of each key column.  The
 *             natural join equates equal ids.  Every id must occur in at least two
 *             relations (a key attribute is a join attribute).
 *   key_cols  host array [n_keys] of pointers, each to n_rows keys of key_type.
 *   n_data    N_i >= 0 data columns; sum over relations must be in [1, 1024].
 *   data      n_rows x n_data float64 matrix, element (r, c) at
 *             data[c*ld + r] (FIGARO_COL_MAJOR, ld >= n_rows) or data[r*ld + c]
 *             (FIGARO_ROW_MAJOR, ld >= n_data).                                       */
typedef struct figaro_relation {
  int64_t n_rows;
  int32_t n_keys;
  int32_t key_type;
  const int32_t* key_attr;
  const void* const* key_cols;
  int32_t n_data;
  int32_t layout;
  int64_t ld;
  const double* data;
} figaro_relation;

/* The database and its join tree tau (§2 "Input"): parent[i] is the parent of
 * relation i, -1 for the single root.  Host memory, read only during figaro_plan. */
typedef struct figaro_join_tree {
  int32_t n_rel;
  const figaro_relation* rels;
  const int32_t* parent;
} figaro_join_tree;

/* Options.  Initialise with figaro_default_options.
 *   precision        FIGARO_PREC_FP64: every step in float64.  FIGARO_PREC_MIXED:
 *                    counts exact; head/tail prefix sums in double-float arithmetic
 *                    (two floats, about 46 bits) with float32 tail rows; the TSQR leaf
 *                    tiles and tree levels of every R0 block in float32; the final QR
 *                    of the stacked block triangles, R, SVD and PCA in float64.
 *                    FIGARO_PREC_MIXED_REFINED: the mixed path followed by one
 *                    CholeskyQR2-style correction (the paper has none): A^T A = R0^T R0
 *                    (Theorem of §6) is accumulated in double-float arithmetic from the
 *                    unrounded tail rows and the float64 blocks, and R = C R~ with
 *                    C = chol(R~^-T A^T A R~^-1) for the mixed R~.  When that Cholesky
 *                    factorisation breaks down (A too ill-conditioned for float32 TSQR),
 *                    R~ is returned as it is and figaro_plan_get_info reports refined = 0.
 *   presorted        1: every relation is already sorted by its key (the order §5
 *                    assumes: attributes shared with the parent first, then the rest,
 *                    each part in ascending attribute id, values ascending); the sort
 *                    is skipped and the order is verified (FIGARO_ERR_NOT_SORTED).
 *   require_reduced  1: fail with FIGARO_ERR_NOT_REDUCED when a tuple does not join
 *                    (the paper assumes fully reduced input, §2); 0 (default): such
 *                    tuples are given weight 0, which is exact since they are not in A.
 *   mem              FIGARO_MEM_DEVICE or FIGARO_MEM_HOST (see the conventions).
 *   stage_timing     1: time every stage with CUDA events (figaro_stage_times).
 *   gradients        1: also hold the workspace of figaro_backward (device memory only).
 *   leaf             FIGARO_LEAF_HOUSEHOLDER (default): Householder TSQR leaves; on
 *                    mixed plans the float leaf of blocks with 33-112 columns runs on the
 *                    5th-generation tensor cores (128-row chunks, 16-column panels in
 *                    registers, both compact-WY products by tcgen05.mma on bf16 triples
 *                    with f32 accumulation in tensor memory).  FIGARO_LEAF_TCGEN05: the
 *                    same, named explicitly.  FIGARO_LEAF_MMA_SYNC: mixed plans fold their
 *                    33-256-column blocks with split-tf32 mma.sync panel updates instead
 *                    (the earlier float leaf; same accuracy class, slower).
 *                    FIGARO_LEAF_GIVENS: TSQR leaves of blocks with <= 16 columns by
 *                    per-thread Givens rotations on 32-row chunks, skipping exact zeros
 *                    (the paper's THIN flavour, for very sparse blocks; wider blocks as
 *                    the default), in float64 on both precisions.
 *   workspace_limit_mib  0 (default): no limit; otherwise figaro_plan fails with
 *                    FIGARO_ERR_NOMEM, allocating nothing, when the plan's device workspace
 *                    would exceed this many MiB (a memory budget for callers that share
 *                    the device).
 *   svd_max_sweeps   0 (default): 40; otherwise the largest number of Jacobi sweeps of
 *                    figaro_svd / figaro_pca / figaro_pca_centered before they give up
 *                    with FIGARO_ERR_TIMEOUT (not converged).
 *   fuse_tails       0 (default): every tails block is written to device memory and then
 *                    triangularised by the TSQR leaf.  1: the tails of a relation with at
 *                    most 32 data columns (Def. "Head and Tail", Alg. 2) are formed in
 *                    registers inside the TSQR leaf (§7 step 1) and never stored (not on
 *                    FIGARO_PREC_MIXED_REFINED plans, nor under FIGARO_LEAF_GIVENS for
 *                    blocks of <= 16 columns); the same R up to rounding, less device
 *                    memory, about as fast (both halves are bound by arithmetic issue, not
 *                    by memory bandwidth).  Any other value: INVALID_ARG.
 *   autotune         0 (default): every TSQR block's leaf tiles, chunk heights, blocks per
 *                    SM, chunks per leaf triangle and tree fan follow the planner's rules
 *                    (width, precision, shared-memory budget).  1: figaro_plan times a few
 *                    candidate plans per block (the rule's among them) on synthetic rows
 *                    of the block's width and row bound (at most 2^30 cells and
 *                    rows x width^2 <= 2^37) and keeps the fastest; results are cached
 *                    per (precision, leaf, width, row bucket)
 *                    for the process, so equal shapes are tuned once.  The same R up to
 *                    rounding (the float path keeps its bound of 16 chunks per leaf
 *                    triangle).  Any other value: INVALID_ARG.                        */
typedef struct figaro_options {
  int32_t precision;
  int32_t presorted;
  int32_t require_reduced;
  int32_t mem;
  int32_t stage_timing;
  int32_t gradients;
  int32_t leaf;
  int32_t workspace_limit_mib;
  int32_t svd_max_sweeps;
  int32_t fuse_tails;
  int32_t autotune;
  int32_t reserved[5];
} figaro_options;

typedef struct figaro_plan_s* figaro_plan_t;

/* Sizes of a plan and of its most recent figaro_qr_r call. */
typedef struct figaro_plan_info {
  int32_t n_rel;
  int32_t n_cols;              /* N, the order of R                                   */
  int64_t input_cells;         /* sum_i M_i (N_i + K_i)                               */
  int64_t input_bytes;         /* bytes of keys and data read per call                */
  int64_t workspace_bytes;     /* device workspace held by the plan                   */
  int64_t r0_rows;             /* rows of R0 after the last call (<= sum_i M_i)       */
  int64_t launches;            /* kernels launched by the last compute call           */
  double tsqr_leaf_flops;      /* algorithmic flops of the TSQR leaf tiles, last call */
  int32_t refined;             /* FIGARO_PREC_MIXED_REFINED: 1 if the last call refined R */
  int32_t reserved;
} figaro_plan_info;

/* Fill *opt with the defaults (FP64, not presorted, reduce, device memory, no timing). */
void figaro_default_options(figaro_options* opt);

/* Validate the database and join tree, scan the key ranges and allocate the device
 * workspace (sized from the bound of the Theorem of §6: R0 has at most sum M_i rows).
 * Key ranges are fixed here: later calls fail with FIGARO_ERR_KEY_RANGE if a key
 * leaves them.  The relation pointers are recorded and read again by every compute
 * call.  Blocks the host until the key-range scan is done.
 * Errors: INVALID_ARG, INVALID_TREE, UNSUPPORTED (more than 64 bits of packed key in
 * one relation, sizes above the limits), NOMEM, CUDA.  *out is NULL on failure.    */
int figaro_plan(const figaro_join_tree* tree, const figaro_options* opt, void* stream,
                figaro_plan_t* out);

/* R (§2 "Output"): sort and segment every relation by key, compute the count
 * aggregates (Alg. 3), the heads and tails (Alg. 4 with Alg. 2) and triangularize R0
 * with a tall-skinny QR (§7).  Writes the N x N upper-triangular R, row-major with
 * leading dimension ldr >= N, normalised to a non-negative diagonal (§2: unique for
 * full rank); entries below the diagonal are written as 0.
 * Errors: INVALID_ARG, NOT_REDUCED, OVERFLOW, KEY_RANGE, NOT_SORTED, CUDA.        */
int figaro_qr_r(figaro_plan_t plan, double* R, int64_t ldr);

/* Singular values and right singular vectors of A (§8.2: those of R).  Computes R as
 * figaro_qr_r does, then a one-sided Jacobi SVD of R in float64.  sigma[N] is
 * descending; V is N x N row-major, column j the j-th right singular vector, each
 * column signed so that its largest-magnitude entry is positive.  R may be NULL; if
 * not, R is also written (row-major, leading dimension N). */
int figaro_svd(figaro_plan_t plan, double* sigma, double* V, double* R);

/* Top-k principal components of A (§8.3, data not centred, as in the paper's
 * experiments): components is N x k row-major (column j = j-th component, the
 * right singular vector of the j-th largest singular value), eigvals[k] = sigma^2.
 * 1 <= k <= N. */
int figaro_pca(figaro_plan_t plan, int32_t k, double* components, double* eigvals);

/* Asynchronous figaro_qr_r: enqueues the same work (with host memory: the input copies,
 * the pipeline and the copy of R back, which needs pinned R) on the plan's stream and
 * returns; figaro_plan_sync waits for it and reports its status.  The inputs and R must
 * stay untouched until then.  Two plans on different streams can overlap one call's
 * transfers with the other's computation.                                              */
int figaro_qr_r_async(figaro_plan_t plan, double* R, int64_t ldr);
int figaro_plan_sync(figaro_plan_t plan);

/* Projections of the join matrix, A X (§8.1-8.3 express Q = A R^-1, U = A V Sigma^-1 and
 * the principal-component scores A V_k through R and its SVD), at the data of the last
 * figaro_qr_r / figaro_svd / figaro_pca call; their row count is the join size, so they
 * are for joins that fit in memory.  The join rows come in a fixed order: the root's
 * tuples in sorted-key order; below a tuple, the combinations of its children's subtrees
 * in mixed radix (first child most significant); inside a child's key group, its tuples
 * in sorted order.
 *   mode   FIGARO_PROJ_X (A X for the caller's X: device, N x k row-major, ld ldx),
 *          FIGARO_PROJ_Q (Q = A R^-1, k = N), FIGARO_PROJ_U (the first k columns of
 *          U = A V Sigma^-1), FIGARO_PROJ_SCORES (A V_k, the top-k PCA scores).
 *   R      device, N x N row-major (ld ldr): the R of that call.
 *   out    device, rows x k row-major (ld ldo >= k).  *rows (if not NULL) receives the
 *          join size; a join larger than max_rows is FIGARO_ERR_UNSUPPORTED (nothing is
 *          written).  A zero diagonal of R (Q) or a zero singular value (U) is
 *          FIGARO_ERR_SINGULAR.  Device memory only; synchronous.
 * figaro_join_size: |J| at the data of the last call (exact).                           */
enum { FIGARO_PROJ_X = 0, FIGARO_PROJ_Q = 1, FIGARO_PROJ_U = 2, FIGARO_PROJ_SCORES = 3 };
int figaro_join_size(figaro_plan_t plan, uint64_t* rows);
int figaro_project(figaro_plan_t plan, int32_t mode, const double* R, int64_t ldr, const double* X, int64_t ldx,
                   int32_t k, double* out, int64_t ldo, int64_t max_rows, int64_t* rows);

/* Centred PCA (not in the paper, whose experiments do not centre): the top-k eigenvectors
 * and eigenvalues of the scatter matrix of the centred join rows,
 * (A - 1 mu^T)^T (A - 1 mu^T) = R^T R - |J| mu mu^T, mu the column means over the join and
 * |J| its row count.  The column sums come from the heads and Phi_circ (sum over the
 * groups of Phi_circ(g) S(g)), |J| from the root's full_join_size (Alg. 3), then the
 * one-sided Jacobi SVD of the N x N scatter matrix (symmetric positive semi-definite: its
 * singular values are its eigenvalues).  components: N x k row-major; eigvals: k values,
 * descending (not divided by |J|).  Same memory rules as figaro_pca.                  */
int figaro_pca_centered(figaro_plan_t plan, int32_t k, double* components, double* eigvals);

/* Gradient of a loss L(R) with respect to every relation's data columns, at the data of
 * the last figaro_qr_r / figaro_svd / figaro_pca call on this plan (made with
 * gradients = 1 and mem = FIGARO_MEM_DEVICE).  The paper does not differentiate R; with
 * Rbar = dL/dR (only its upper triangle matters), R of full column rank, and
 * W = R^-1 copyltu(R Rbar^T) R^-T (copyltu mirrors the lower triangle), dL/dA = A W for
 * the join matrix A, and the gradient for tuple t of relation k is
 * m(t)^T W[:, Y_k], m(t) the sum of the join rows that contain t (Phi_circ(t) y_t on Y_k,
 * sums from messages over the join tree, counted with Alg. 3's aggregates, elsewhere).
 *   R      device, N x N row-major (ldr >= N): the R that call returned.
 *   Rbar   device, N x N row-major (ldb >= N).
 *   grads  host array of n_rel device pointers: relation i's gradient, column-major
 *          M_i x N_i with leading dimension ldg[i] >= M_i, in the input row order
 *          (NULL for a relation without data columns).
 * Errors: FIGARO_ERR_SINGULAR (a zero diagonal entry of R), FIGARO_ERR_UNSUPPORTED (plan
 * without gradients or in host-memory mode).  Sums are formed with atomics: results are
 * accurate to rounding but not bitwise reproducible.  Synchronous.                     */
int figaro_backward(figaro_plan_t plan, const double* R, int64_t ldr, const double* Rbar, int64_t ldb,
                    double* const* grads, const int64_t* ldg);

/* Batches of independent instances (many joins, each with its own plan) as one CUDA
 * graph: every plan's R pipeline, and with k[i] > 0 its Jacobi SVD and top-k principal
 * components, become independent branches of one graph that figaro_batch_run launches
 * at once, so that small and uneven instances overlap on the GPU.  The paper treats one
 * join at a time; batching is not part of it.
 *   plans       n distinct plans (device memory, stage_timing = 0).  Their inputs are
 *               read at every run; a plan must not be used elsewhere while a run is in
 *               flight.
 *   R[i]        device, N_i x N_i row-major (ld N_i): instance i's R.
 *   components, eigvals, k   NULL, or per instance: k[i] in [0, N_i]; when k[i] > 0,
 *               components[i] (device, N_i x k[i] row-major) and eigvals[i] (device, k[i])
 *               as figaro_pca writes them.
 * figaro_batch_run launches the graph and waits; status (NULL or n entries) receives each
 * instance's error word, and the first non-zero one is returned.  figaro_batch_launches
 * is the number of kernels one run launches.                                          */
typedef struct figaro_batch_s* figaro_batch_t;
int figaro_batch_create(int32_t n, const figaro_plan_t* plans, double* const* R, double* const* components,
                        double* const* eigvals, const int32_t* k, figaro_batch_t* out);
int figaro_batch_run(figaro_batch_t batch, int32_t* status);
int64_t figaro_batch_launches(figaro_batch_t batch);
int figaro_batch_destroy(figaro_batch_t batch);

/* Release the plan's workspace (waits for its stream).  NULL is accepted. */
int figaro_plan_destroy(figaro_plan_t plan);

/* Sizes of the plan and of its last call. */
int figaro_plan_get_info(figaro_plan_t plan, figaro_plan_info* info);

/* Stage times in milliseconds summed over the compute calls since the last reset,
 * when the plan was made with stage_timing = 1 (else zeros).  Stages:
 *   0 key packing and radix sort, 1 segmentation, 2 count aggregates (Alg. 3),
 *   3 heads and tails of the relations (Alg. 4 heads_and_tails),
 *   4 join of children and projection (Alg. 4 process_and_join_children,
 *     project_away_join_attributes, root), 5 TSQR leaf tiles, 6 TSQR tree and final
 *   QR, 7 SVD.  counts[s] is the number of kernel launches of stage s in the same
 *   period.  Returns the number of stages (8) or a negative status.                */
int figaro_stage_times(figaro_plan_t plan, double* ms, int64_t* counts, int32_t n);
int figaro_reset_stage_times(figaro_plan_t plan);

/* Per block of R0 (§7: for every relation in order, its tails block if it has data
 * columns, then its generalized-tail block (inner relations) or the root block): the
 * time of the block's TSQR leaf launches in milliseconds summed since the last reset
 * (stage_timing = 1 only, else 0), its column count and its row count in the last
 * call.  Any of the three host arrays may be NULL; at most `max` entries are written.
 * A measurement aid (the paper has no counterpart).  Returns the number of blocks or a
 * negative status.                                                                   */
int figaro_block_times(figaro_plan_t plan, int32_t max, double* leaf_ms, int32_t* n_cols, int64_t* rows);

/* Copy an intermediate array of relation `rel` from the last compute call to host
 * memory, for tests and diagnostics (a synchronous copy of at most `bytes` bytes).
 * Returns the number of bytes the array holds (>= 0) or a negative status.
 *   FIGARO_DBG_SIZES     int64[8]: M, G (groups of X_i), P (groups of X_p), tail
 *                        rows, generalized-tail rows, root rows, K, N_sub
 *   FIGARO_DBG_PERM      int32[M]: row of the input at each sorted position
 *   FIGARO_DBG_GROUP_OFF int32[G+1]: first sorted position of every group
 *   FIGARO_DBG_COUNTS    uint64[4*G]: rows_per_key, Theta_down, full_join_size,
 *                        Phi_circ of every group (group-major)
 *   FIGARO_DBG_PCOUNTS   uint64[2*P]: Phi_down, Phi_up of every X_p group
 *   FIGARO_DBG_TAILS     float64[(M-G) x N_i] column-major: sqrt(Phi_circ) T(S^{x})
 *                        of every group, groups in key order (INVALID_ARG when the
 *                        plan formed them inside the TSQR leaf: see fuse_tails)
 *   FIGARO_DBG_HEADS     float64[G x N_i] column-major: H(S^{x}) of every group
 *   FIGARO_DBG_GEN_TAILS float64[(G-P) x N_sub] column-major: generalized tails of
 *                        the projection (internal non-root relations)
 *   FIGARO_DBG_DATA      float64[P x N_sub] column-major: the generalized heads
 *                        passed to the parent (internal non-root relations)
 *   FIGARO_DBG_ROOT_ROWS float64[G x N] column-major: the root's Data rows
 * TAILS and GEN_TAILS hold the float64 rows of FIGARO_PREC_FP64 plans; mixed plans keep
 * their tail rows in float32 (GEN_TAILS of FIGARO_PREC_MIXED_REFINED plans stay float64)
 * and those arrays are not read by them.                                              */
enum {
  FIGARO_DBG_SIZES = 0, FIGARO_DBG_PERM = 1, FIGARO_DBG_GROUP_OFF = 2, FIGARO_DBG_COUNTS = 3,
  FIGARO_DBG_PCOUNTS = 4, FIGARO_DBG_TAILS = 5, FIGARO_DBG_HEADS = 6, FIGARO_DBG_GEN_TAILS = 7,
  FIGARO_DBG_DATA = 8, FIGARO_DBG_ROOT_ROWS = 9
};
int64_t figaro_debug_read(figaro_plan_t plan, int32_t rel, int32_t what, void* dst, int64_t bytes);

/* SVD of a given N x N matrix R (row-major, leading dimension ldr >= N, device memory)
 * without any device allocation: the paper has no counterpart; this entry point exists for
 * callers that cannot allocate device memory when they need the SVD -- for example a
 * process whose device memory is entirely reserved by its own pool allocator, or a
 * latency-critical loop in which the implicit synchronisation of an allocation is not
 * acceptable.  The caller passes R and the outputs: sigma[N] (descending) and V (N x N
 * row-major, column j the j-th right singular vector, signed so that its largest-magnitude
 * entry is positive), both device pointers, exactly as figaro_svd returns them.
 * Work arrays live in one fixed device array of 2 * 256 * 256 doubles plus an error word
 * (about 1 MiB), defined in the library and held by every GPU that loads it until the
 * process exits; N larger than 256 is rejected with FIGARO_ERR_UNSUPPORTED before any
 * device work.  Every call looks up that array's device address with the calling thread's
 * current device (a host query, made before anything is enqueued).  All calls share the
 * array: calls whose executions overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  Enqueues on `stream` and waits for it before
 * returning; because of that wait, a `stream` that is being captured is refused with
 * FIGARO_ERR_UNSUPPORTED before anything is enqueued.  figaro_last_error describes the
 * failure of the last call on this thread.  Errors: INVALID_ARG, UNSUPPORTED, TIMEOUT (no
 * convergence in 40 sweeps), CUDA. */
int figaro_svd_from_r_static(const double* R, int64_t ldr, int32_t n, double* sigma, double* V,
                             void* stream);

/* Measurement aid, not part of the paper's method: the FP64 FMA rate of the current
 * device in TFLOP/s (2 flops per FMA), from five launches of a kernel whose threads run
 * eight independent FMA chains each (64 warps per SM), timed with CUDA events on
 * `stream` after one warm-up launch; waits for the stream.  It is the measured ceiling
 * that the benchmark quotes the FP64-pipe-bound kernels against.  Errors: INVALID_ARG, CUDA. */
int figaro_fp64_fma_rate(double* tflops, void* stream);

/* Name of a status code (static storage). */
const char* figaro_error_string(int status);

/* Details of the most recent failure on the calling thread ("" if none). */
const char* figaro_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FIGARO_H */
